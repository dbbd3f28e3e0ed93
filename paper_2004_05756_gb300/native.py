"""Thin Python binding of libtopo.so (include/topo.h): the same entry points, argument
marshalling only. Device arrays are torch CUDA tensors (PyTorch owns device memory and
streams); every step of the computation runs in the library's CUDA kernels.

There is no fallback: if libtopo.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libtopo.so")

TOPO_OK, TOPO_ERR_INVALID, TOPO_ERR_OOM, TOPO_ERR_NOT_CONVERGED, TOPO_ERR_NOT_SPD, TOPO_ERR_TIMEOUT, TOPO_ERR_CUDA = range(7)
STATUS_NAMES = {0: "TOPO_OK", 1: "TOPO_ERR_INVALID", 2: "TOPO_ERR_OOM", 3: "TOPO_ERR_NOT_CONVERGED",
                4: "TOPO_ERR_NOT_SPD", 5: "TOPO_ERR_TIMEOUT", 6: "TOPO_ERR_CUDA"}
TOPO_FP64, TOPO_FP32_REFINED, TOPO_FP32_BF16KE_REFINED = 0, 1, 2
PREC = {"fp64": TOPO_FP64, "fp32": TOPO_FP32_REFINED, "fp32_bf16ke": TOPO_FP32_BF16KE_REFINED}
(TOPO_PARAM_INNER_RTOL, TOPO_PARAM_MAX_OUTER, TOPO_PARAM_WAIT_CYCLES, TOPO_PARAM_ROM_REFINE,
 TOPO_PARAM_TILE_X, TOPO_PARAM_PCG_BLOCKS_PER_SM, TOPO_PARAM_INNER_CAP, TOPO_PARAM_HDM_KERNEL,
 TOPO_PARAM_PCG_MAX_CTAS, TOPO_PARAM_ROM_TENSOR, TOPO_PARAM_APPLY_STAGES, TOPO_PARAM_PCG_POLY,
 TOPO_PARAM_PCG_MG, TOPO_PARAM_MG_DEGREE, TOPO_PARAM_MG_SINGLE_NODES, TOPO_PARAM_FILTER,
 TOPO_PARAM_HELMHOLTZ_R, TOPO_PARAM_ROM_ASSEMBLY) = range(18)

# Every entry point declared in include/topo.h (checked by the tests).
EXPORTS = ["topo_create", "topo_destroy", "topo_last_error", "topo_set_param", "topo_check", "topo_sizes",
           "topo_filter", "topo_apply_K", "topo_solve_hdm", "topo_rom_build", "topo_rom_solve",
           "topo_rom_error", "topo_compliance_grad", "topo_launch_count", "topo_rom_elem",
           "topo_rom_solve_elem", "topo_rom_solve_elem_noalloc", "topo_rom_eval_batch", "topo_batch_create",
           "topo_batch_destroy",
           "topo_batch_last_error", "topo_batch_context", "topo_batch_solve_hdm", "topo_batch_filter",
           "topo_batch_compliance_grad", "topo_batch_rom_solve_elem", "topo_tr_init", "topo_tr_project",
           "topo_tr_trials", "topo_tr_select", "topo_tr_update", "topo_rom_pod", "topo_output_grad",
           "topo_rom_rhs", "topo_sigma_min", "topo_rom_assemble_batch"]


class TopoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class topo_problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("E0", ctypes.c_double), ("Emin", ctypes.c_double), ("nu", ctypes.c_double),
                ("penal", ctypes.c_double), ("rmin", ctypes.c_double),
                ("fixed_dof_mask", ctypes.POINTER(ctypes.c_ubyte))]


class topo_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("relres", ctypes.c_double),
                ("status", ctypes.c_int), ("floor", ctypes.c_double), ("poly", ctypes.c_int),
                ("mg_levels", ctypes.c_int), ("fallback", ctypes.c_int)]


class topo_tr_state(ctypes.Structure):
    """Host image of the device-resident trust-region state (128 bytes)."""
    _fields_ = [(n, ctypes.c_double) for n in ("delta", "delta_max", "delta_prev", "J_c", "Jk_c", "Jk_hat", "J_hat",
                                               "theta_hat", "step", "ratio", "gtd", "pad0")] + \
               [(n, ctypes.c_int) for n in ("sel", "inside", "accepted", "iter")] + [("pad1", ctypes.c_int * 4)]


class topo_tr_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("gamma1", "gamma2", "eta1", "eta2", "grow", "c1")]


TR_STATE_BYTES = ctypes.sizeof(topo_tr_state)


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libtopo.so and declare the C signatures. Raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtopo.so not built ({path}); run paper_2004_05756_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "topo_create": ([ctypes.POINTER(topo_problem), P, ctypes.POINTER(P)], I),
        "topo_destroy": ([P], I),
        "topo_last_error": ([P], ctypes.c_char_p),
        "topo_set_param": ([P, I, D], I),
        "topo_check": ([P], I),
        "topo_sizes": ([P, ctypes.POINTER(LL), ctypes.POINTER(LL), ctypes.POINTER(LL)], I),
        "topo_filter": ([P, P, P, I], I),
        "topo_apply_K": ([P, P, P, P, I, I, I], I),
        "topo_solve_hdm": ([P, P, P, P, I, I, D, I, I, ctypes.POINTER(topo_solve_info)], I),
        "topo_rom_build": ([P, P, P, I, I, P, ctypes.POINTER(I), P, P, P], I),
        "topo_rom_solve": ([P, P, P, I, I, P, P, P, P, I], I),
        "topo_rom_error": ([P, P, P, I, I, P, P, P, P], I),
        "topo_compliance_grad": ([P, P, P, I, I, P, P, P, P], I),
        "topo_launch_count": ([ctypes.POINTER(LL)], I),
        "topo_rom_elem": ([P, P, I, I, P], I),
        "topo_rom_solve_elem": ([P, P, P, I, P, P, P, P], I),
        "topo_rom_solve_elem_noalloc": ([P, P, P, I, P, P, P, P], I),
        "topo_rom_eval_batch": ([P, I, P, I, I, P, P, I, I, P, P, P, P, P, P], I),
        "topo_rom_assemble_batch": ([P, I, P, LL, P, I, P], I),
        "topo_batch_create": ([ctypes.POINTER(topo_problem), I, P, ctypes.POINTER(P)], I),
        "topo_batch_destroy": ([P], I),
        "topo_batch_last_error": ([P], ctypes.c_char_p),
        "topo_batch_context": ([P, I, ctypes.POINTER(P)], I),
        "topo_batch_solve_hdm": ([P, P, P, P, P, P, D, I, ctypes.POINTER(topo_solve_info)], I),
        "topo_batch_filter": ([P, P, P, I], I),
        "topo_batch_compliance_grad": ([P, P, P, P, P, P, P, P, P], I),
        "topo_batch_rom_solve_elem": ([P, P, P, P, P, P, P, P], I),
        "topo_tr_init": ([P, P, P, D, D, P], I),
        "topo_rom_pod": ([P, P, I, I, I, I, P, P, I, P], I),
        "topo_output_grad": ([P, P, P, P, I, I, P, P, P, P], I),
        "topo_rom_rhs": ([P, P, I, I, P, P], I),
        "topo_sigma_min": ([P, P, I, D, P], I),
        "topo_tr_project": ([P, P, P, D, I, D, P, P], I),
        "topo_tr_trials": ([P, I, P, P, P, I], I),
        "topo_tr_select": ([P, P, ctypes.POINTER(topo_tr_params), I, P, P, P, P, I, P, I, I, P, P, P], I),
        "topo_tr_update": ([P, P, ctypes.POINTER(topo_tr_params), P, P, P, P, P, P, P, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def launch_count() -> int:
    """Kernel launches issued by libtopo so far in this process."""
    n = ctypes.c_longlong(0)
    load().topo_launch_count(ctypes.byref(n))
    return int(n.value)


def _ptr(t) -> int | None:
    """Device address of a CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise TypeError("libtopo arrays must be CUDA tensors")
    return t.data_ptr()


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Topo:
    """One libtopo context (one problem on one device and stream). Method names follow the
    C entry points; each method checks dtypes/shapes and forwards raw pointers."""

    def __init__(self, problem, stream=None):
        self.lib = load()
        self.problem = problem
        mask = np.ascontiguousarray(problem.fixed, dtype=np.uint8)
        self._mask = mask
        pr = topo_problem(problem.dim, problem.nx, problem.ny, problem.nz if problem.dim == 3 else 1,
                          problem.E0, problem.Emin, problem.nu, problem.penal, problem.rmin,
                          mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        self.stream = stream
        h = ctypes.c_void_p()
        st = self.lib.topo_create(ctypes.byref(pr), _stream_handle(stream), ctypes.byref(h))
        if st != TOPO_OK:
            raise TopoError(st, "topo_create failed")
        self.h = h
        self.N = problem.ndof
        self.Ne = problem.nel

    # -- plumbing ------------------------------------------------------------------------
    def _chk(self, st: int, what: str):
        if st != TOPO_OK:
            raise TopoError(st, f"{what}: {self.lib.topo_last_error(self.h).decode(errors='replace')}")

    @classmethod
    def borrowed(cls, handle, problem, stream=None):
        """A view of a context the caller does not own (an instance of a topo_batch): the same
        methods, and close() leaves the context to its owner."""
        t = cls.__new__(cls)
        t.lib = load()
        t.problem = problem
        t.stream = stream
        t.h = handle
        t.N = problem.ndof
        t.Ne = problem.nel
        t._borrowed = True
        return t

    def close(self):
        if getattr(self, "h", None):
            if not getattr(self, "_borrowed", False):
                self.lib.topo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def topo_set_param(self, which: int, value: float):
        self._chk(self.lib.topo_set_param(self.h, which, float(value)), "topo_set_param")

    def topo_check(self):
        self._chk(self.lib.topo_check(self.h), "topo_check")

    # -- the hot path ---------------------------------------------------------------------
    def topo_filter(self, x, out, adjoint: bool = False):
        self._chk(self.lib.topo_filter(self.h, _ptr(x), _ptr(out), int(adjoint)), "topo_filter")
        return out

    def topo_apply_K(self, rho, V, Y, prec: str = "fp64"):
        m, ld = _cols(V, self.N)
        self._chk(self.lib.topo_apply_K(self.h, _ptr(rho), _ptr(V), _ptr(Y), m, ld, PREC[prec]), "topo_apply_K")
        return Y

    def topo_solve_hdm(self, rho, F, U, rtol: float = 1e-8, maxit: int = 100000, prec: str = "fp64",
                       info: bool = True):
        m, ld = _cols(F, self.N)
        inf = topo_solve_info()
        st = self.lib.topo_solve_hdm(self.h, _ptr(rho), _ptr(F), _ptr(U), m, ld, float(rtol), int(maxit),
                                     PREC[prec], ctypes.byref(inf) if info else None)
        if st not in (TOPO_OK, TOPO_ERR_NOT_CONVERGED):
            self._chk(st, "topo_solve_hdm")
        return dict(iters=inf.iters, outer=inf.outer, relres=inf.relres, status=inf.status, poly=inf.poly,
                    floor=inf.floor, mg_levels=inf.mg_levels, fallback=inf.fallback) if info else None

    def topo_rom_build(self, rho, Usnap, Phi, H, b, f):
        m, ld = _cols(Usnap, self.N)
        k = ctypes.c_int(0)
        self._chk(self.lib.topo_rom_build(self.h, _ptr(rho), _ptr(Usnap), m, ld, _ptr(Phi), ctypes.byref(k),
                                          _ptr(H), _ptr(b), _ptr(f)), "topo_rom_build")
        return k.value

    def topo_rom_solve(self, rho, Phi, k: int, b, H_work, yhat, Jk, prec: str = "fp64"):
        ld = _ld(Phi, self.N)
        self._chk(self.lib.topo_rom_solve(self.h, _ptr(rho), _ptr(Phi), int(k), ld, _ptr(b), _ptr(H_work),
                                          _ptr(yhat), _ptr(Jk), PREC[prec]), "topo_rom_solve")

    def topo_rom_pod(self, U, n: int, Pod, sigma, skip: int = -1, append=None):
        """U: (m, ld) snapshot block; Pod: (n + (append is not None), ldp)."""
        m, ld = _cols(U, self.N)
        _, ldp = _cols(Pod, self.N)
        self._chk(self.lib.topo_rom_pod(self.h, _ptr(U), m, ld, int(skip), int(n), _ptr(append), _ptr(Pod), ldp,
                                        _ptr(sigma)), "topo_rom_pod")

    def topo_rom_elem(self, Phi, k: int, Hel):
        ld = _ld(Phi, self.N)
        self._chk(self.lib.topo_rom_elem(self.h, _ptr(Phi), int(k), ld, _ptr(Hel)), "topo_rom_elem")
        return Hel

    def topo_rom_solve_elem(self, rho, Hel, k: int, b, H_work, yhat, Jk):
        self._chk(self.lib.topo_rom_solve_elem(self.h, _ptr(rho), _ptr(Hel), int(k), _ptr(b), _ptr(H_work),
                                               _ptr(yhat), _ptr(Jk)), "topo_rom_solve_elem")

    def topo_rom_solve_elem_noalloc(self, rho, Hel, k: int, b, H_work, yhat, Jk):
        self._chk(self.lib.topo_rom_solve_elem_noalloc(self.h, _ptr(rho), _ptr(Hel), int(k), _ptr(b), _ptr(H_work),
                                                       _ptr(yhat), _ptr(Jk)), "topo_rom_solve_elem_noalloc")

    def topo_rom_eval_batch(self, psi, Hel, Phi, k: int, b, f, Jk, resnorm, yhat=None, dpsi=None,
                            filtered: bool = True):
        """psi: (R, ldp) tensor of designs (rows = candidates); Jk (R,), resnorm (R, 2), yhat (R, k),
        dpsi (R, ldp) like psi."""
        R = int(psi.shape[0]) if psi.dim() == 2 else 1
        ldp = int(psi.stride(0)) if psi.dim() == 2 and R > 1 else int(self.Ne)
        if dpsi is not None and dpsi.dim() == 2 and R > 1 and int(dpsi.stride(0)) != ldp:
            raise ValueError("dpsi must have the stride of psi")
        ld = _ld(Phi, self.N)
        self._chk(self.lib.topo_rom_eval_batch(self.h, R, _ptr(psi), ldp, 1 if filtered else 0, _ptr(Hel), _ptr(Phi),
                                               int(k), ld, _ptr(b), _ptr(f), _ptr(Jk), _ptr(resnorm), _ptr(yhat),
                                               _ptr(dpsi)), "topo_rom_eval_batch")

    def topo_rom_assemble_batch(self, E, Hel, k: int, H):
        """E: (R, ldE) moduli rows (N_e + 1 used each); H: R * k * k doubles."""
        R = int(E.shape[0]) if E.dim() == 2 else 1
        ldE = int(E.stride(0)) if E.dim() == 2 and R > 1 else int(self.Ne) + 1
        self._chk(self.lib.topo_rom_assemble_batch(self.h, R, _ptr(E), ldE, _ptr(Hel), int(k), _ptr(H)),
                  "topo_rom_assemble_batch")

    def topo_rom_error(self, rho, Phi, k: int, yhat, f, resnorm, uk=None):
        ld = _ld(Phi, self.N)
        self._chk(self.lib.topo_rom_error(self.h, _ptr(rho), _ptr(Phi), int(k), ld, _ptr(yhat), _ptr(f),
                                          _ptr(resnorm), _ptr(uk)), "topo_rom_error")

    def topo_compliance_grad(self, rho, U, F, J, dc_rho, dc_psi=None):
        m, ld = _cols(U, self.N)
        self._chk(self.lib.topo_compliance_grad(self.h, _ptr(rho), _ptr(U), m, ld, _ptr(F), _ptr(J),
                                                _ptr(dc_rho), _ptr(dc_psi)), "topo_compliance_grad")

    def topo_output_grad(self, rho, U, Lam, L, J, dc_rho, dc_psi=None):
        m, ld = _cols(U, self.N)
        m2, ld2 = _cols(Lam, self.N)
        m3, ld3 = _cols(L, self.N)
        if (m2, ld2) != (m, ld) or (m3, ld3) != (m, ld):
            raise ValueError("U, Lam and L must share their shape and leading dimension")
        self._chk(self.lib.topo_output_grad(self.h, _ptr(rho), _ptr(U), _ptr(Lam), m, ld, _ptr(L), _ptr(J),
                                            _ptr(dc_rho), _ptr(dc_psi)), "topo_output_grad")

    def topo_rom_rhs(self, Phi, k: int, v, out):
        self._chk(self.lib.topo_rom_rhs(self.h, _ptr(Phi), int(k), _ld(Phi, self.N), _ptr(v), _ptr(out)),
                  "topo_rom_rhs")

    def topo_sigma_min(self, rho, out, steps: int = 30, rtol: float = 1e-10):
        """out (device FP64[4]): estimate, lower bound, theta, Ritz residual."""
        self._chk(self.lib.topo_sigma_min(self.h, _ptr(rho), int(steps), float(rtol), _ptr(out)), "topo_sigma_min")

    # -- trust-region step (Algorithm 2) ----------------------------------------------------
    def topo_tr_init(self, st, f, tau: float, dmax_factor: float, J_c):
        self._chk(self.lib.topo_tr_init(self.h, _ptr(st), _ptr(f), float(tau), float(dmax_factor), _ptr(J_c)),
                  "topo_tr_init")

    def topo_tr_project(self, psi, g, t: float, scaled: bool, vmax: float, out, stats):
        self._chk(self.lib.topo_tr_project(self.h, _ptr(psi), _ptr(g), float(t), 1 if scaled else 0, float(vmax),
                                           _ptr(out), _ptr(stats)), "topo_tr_project")

    def topo_tr_trials(self, psi_c, psi_x, trials):
        """trials: (R, ldt) tensor; row r = psi_c + s_r (psi_x - psi_c)."""
        R, ldt = int(trials.shape[0]), int(trials.stride(0)) if trials.shape[0] > 1 else int(self.Ne)
        self._chk(self.lib.topo_tr_trials(self.h, R, _ptr(psi_c), _ptr(psi_x), _ptr(trials), ldt), "topo_tr_trials")

    def topo_tr_select(self, st, prm, Jk, resnorm, gtd, trials, Phi, k: int, yhat, psi_hat, u_hat):
        R, ldt = int(trials.shape[0]), int(trials.stride(0)) if trials.shape[0] > 1 else int(self.Ne)
        ld = _ld(Phi, self.N)
        self._chk(self.lib.topo_tr_select(self.h, _ptr(st), ctypes.byref(prm), R, _ptr(Jk), _ptr(resnorm), _ptr(gtd),
                                          _ptr(trials), ldt, _ptr(Phi), int(k), ld, _ptr(yhat), _ptr(psi_hat),
                                          _ptr(u_hat)), "topo_tr_select")

    def topo_tr_update(self, st, prm, J_hat, psi_c, psi_hat, u_c, u_hat, g_c, g_hat, u_slot=None):
        self._chk(self.lib.topo_tr_update(self.h, _ptr(st), ctypes.byref(prm), _ptr(J_hat), _ptr(psi_c),
                                          _ptr(psi_hat), _ptr(u_c), _ptr(u_hat), _ptr(g_c), _ptr(g_hat),
                                          _ptr(u_slot)), "topo_tr_update")


def tr_state_tensor():
    """A zeroed device buffer for one topo_tr_state (FP64 view of its 128 bytes)."""
    import torch
    return torch.zeros(TR_STATE_BYTES // 8, dtype=torch.float64, device="cuda")


def tr_state_read(st) -> dict:
    """Copy a device topo_tr_state to the host and decode it (synchronises its stream)."""
    raw = st.detach().cpu().numpy().tobytes()
    h = topo_tr_state.from_buffer_copy(raw)
    return {n: getattr(h, n) for n, _ in topo_tr_state._fields_ if not n.startswith("pad")}


def tr_params(gamma1=0.5, gamma2=1.0, eta1=0.1, eta2=0.75, grow=2.0, c1=1e-4) -> topo_tr_params:
    return topo_tr_params(gamma1, gamma2, eta1, eta2, grow, c1)


def _cols(t, N: int):
    """Column count and leading dimension of an N x m column-major block stored as a torch
    tensor of shape (m, ld) (row c = column c) or a 1-D vector of length >= N."""
    if t.dim() == 1:
        return 1, int(t.shape[0])
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError("column blocks must be (m, ld) tensors with unit stride along ld")
    if t.shape[0] == 1:  # a single column: its stride along dim 0 is meaningless
        return 1, int(t.shape[1])
    return int(t.shape[0]), int(t.stride(0))


def _ld(t, N: int) -> int:
    return _cols(t, N)[1]


def _ptr_array(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = _ptr(t)
    return arr


def _int_array(vals):
    return (ctypes.c_int * len(vals))(*[int(v) for v in vals])


class TopoBatch:
    """Batched form (topo_batch_*): many 2D problems on one stream. Lists of CUDA tensors are
    marshalled into host pointer arrays."""

    def __init__(self, problems, stream=None):
        self.lib = load()
        self.problems = list(problems)
        self._masks = [np.ascontiguousarray(p.fixed, dtype=np.uint8) for p in self.problems]
        arr = (topo_problem * len(self.problems))()
        for i, (p, mk) in enumerate(zip(self.problems, self._masks)):
            arr[i] = topo_problem(p.dim, p.nx, p.ny, 1, p.E0, p.Emin, p.nu, p.penal, p.rmin,
                                  mk.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        h = ctypes.c_void_p()
        st = self.lib.topo_batch_create(arr, len(self.problems), _stream_handle(stream), ctypes.byref(h))
        if st != TOPO_OK:
            raise TopoError(st, "topo_batch_create failed")
        self.h = h
        self.count = len(self.problems)

    def _chk(self, st, what):
        if st != TOPO_OK:
            raise TopoError(st, f"{what}: {self.lib.topo_batch_last_error(self.h).decode(errors='replace')}")

    def context(self, i: int):
        """Topo view of instance i's context (owned by the batch)."""
        c = ctypes.c_void_p()
        self._chk(self.lib.topo_batch_context(self.h, int(i), ctypes.byref(c)), "topo_batch_context")
        return Topo.borrowed(c, self.problems[i])

    def set_param(self, which: int, value: float):
        """topo_set_param on every instance context (e.g. TOPO_PARAM_PCG_MG: 1 runs the batched
        solve with the multigrid preconditioner, 0 with Jacobi)."""
        for i in range(self.count):
            c = ctypes.c_void_p()
            self._chk(self.lib.topo_batch_context(self.h, i, ctypes.byref(c)), "topo_batch_context")
            st = self.lib.topo_set_param(c, int(which), float(value))
            if st != TOPO_OK:
                raise TopoError(st, f"topo_set_param on instance {i}: "
                                    f"{self.lib.topo_last_error(c).decode(errors='replace')}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.topo_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def topo_batch_filter(self, xs, outs, adjoint=False):
        self._chk(self.lib.topo_batch_filter(self.h, _ptr_array(xs), _ptr_array(outs), int(adjoint)), "topo_batch_filter")

    def topo_batch_solve_hdm(self, rhos, Fs, Us, rtol=1e-8, maxit=200000, info=True):
        ms, lds = zip(*[_cols(F, 0) for F in Fs])
        inf = (topo_solve_info * self.count)() if info else None
        st = self.lib.topo_batch_solve_hdm(self.h, _ptr_array(rhos), _ptr_array(Fs), _ptr_array(Us), _int_array(ms),
                                           _int_array(lds), float(rtol), int(maxit), inf)
        if st not in (TOPO_OK, TOPO_ERR_NOT_CONVERGED):
            self._chk(st, "topo_batch_solve_hdm")
        if not info:
            return None
        return [dict(iters=x.iters, relres=x.relres, status=x.status, floor=x.floor, poly=x.poly,
                     mg_levels=x.mg_levels, fallback=x.fallback) for x in inf]

    def topo_batch_compliance_grad(self, rhos, Us, Fs, J, dcs, dpsis=None):
        ms, lds = zip(*[_cols(U, 0) for U in Us])
        self._chk(self.lib.topo_batch_compliance_grad(self.h, _ptr_array(rhos), _ptr_array(Us), _int_array(ms),
                                                      _int_array(lds), _ptr_array(Fs), _ptr(J), _ptr_array(dcs),
                                                      _ptr_array(dpsis) if dpsis is not None else None),
                  "topo_batch_compliance_grad")

    def topo_batch_rom_solve_elem(self, rhos, Hels, ks, bs, Hws, ys, Jk):
        self._chk(self.lib.topo_batch_rom_solve_elem(self.h, _ptr_array(rhos), _ptr_array(Hels), _int_array(ks),
                                                     _ptr_array(bs), _ptr_array(Hws), _ptr_array(ys), _ptr(Jk)),
                  "topo_batch_rom_solve_elem")
