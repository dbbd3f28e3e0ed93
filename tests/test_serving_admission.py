"""Host logic of the serving admission, without a GPU.

- Requests start in arrival order.
- When the earliest waiting request does not fit the memory budget, the least recently used
  idle session is evicted; busy sessions and the requester itself are never chosen.
- A spilled session re-admits its own bytes before its next request runs, and waits while its
  own eviction is still copying.

The server's admission methods run against stand-in sessions whose eviction only records itself.
"""
import threading
import time

from paper_2004_05756_gb300.serving import Request, Server


class StubSession:
    def __init__(self, name, held, last_use, log, busy=False):
        self.name = name
        self.held = held
        self.counted = True
        self.resident = True
        self.busy = busy
        self.evicting = False
        self.last_use = last_use
        self.log = log

    def evict(self):
        self.log.append(("evict", self.name))
        self.resident = False


def _server(budget, slots):
    srv = object.__new__(Server)  # the admission state only: no device, no library
    srv.lock = threading.Condition()
    srv.budget = budget
    srv.in_use = 0
    srv.free_slots = list(range(slots))
    srv.concurrency = 0
    srv.max_concurrency = 0
    srv.sessions = {}
    srv.waiting = []
    srv.evictions = 0
    srv.restores = 0
    srv.evict_ms = []
    srv.restore_ms = []
    return srv


def _req(rid, arrival=0.0):
    return Request(rid=rid, dim=2, shape=(2, 1), seed=0, arrival=arrival)


def _wait_for(cond, timeout=5.0):
    t0 = time.time()
    while not cond():
        assert time.time() - t0 < timeout, "timed out"
        time.sleep(0.001)


def test_evicts_least_recently_used_idle_sessions_only():
    log = []
    srv = _server(budget=100, slots=2)
    A = StubSession("A", 30, last_use=1.0, log=log)
    B = StubSession("B", 30, last_use=2.0, log=log)
    C = StubSession("C", 30, last_use=0.5, log=log, busy=True)  # oldest, but running
    srv.sessions = {0: A, 1: B, 2: C}
    srv.in_use = 90
    slot, admitted = srv._acquire(_req(7), 50)
    assert admitted == 50
    assert log == [("evict", "A"), ("evict", "B")]  # A first (least recent), C never
    assert srv.in_use == 30 + 50 and srv.evictions == 2
    assert not A.counted and not B.counted and C.counted and C.resident


def test_no_eviction_when_the_request_fits():
    log = []
    srv = _server(budget=100, slots=2)
    srv.sessions = {0: StubSession("A", 30, 1.0, log)}
    srv.in_use = 30
    srv._acquire(_req(1), 70)
    assert log == [] and srv.in_use == 100


def test_requests_start_in_arrival_order():
    srv = _server(budget=1000, slots=1)
    first, _ = srv._acquire(_req(99, 0.0), 0)  # holds the only slot
    order = []

    def worker(req):
        slot, _ = srv._acquire(req, 0)
        order.append(req.rid)
        srv._release(slot, 0)

    late = threading.Thread(target=worker, args=(_req(1, arrival=1.0),))
    late.start()
    _wait_for(lambda: len(srv.waiting) == 1)
    early = threading.Thread(target=worker, args=(_req(0, arrival=0.5),))
    early.start()
    _wait_for(lambda: len(srv.waiting) == 2)
    srv._release(first, 0)
    late.join(5)
    early.join(5)
    assert order == [0, 1]


def test_spilled_session_readmits_its_bytes_and_may_evict_others():
    log = []
    srv = _server(budget=100, slots=2)
    S = StubSession("S", 40, last_use=5.0, log=log)
    S.counted = S.resident = False  # spilled earlier
    D = StubSession("D", 70, last_use=0.0, log=log)
    srv.sessions = {0: S, 1: D}
    srv.in_use = 70
    slot, admitted = srv._acquire(_req(3), 0, owner=S)
    assert admitted == 40 and log == [("evict", "D")]
    assert S.busy and S.counted and srv.in_use == 40


def test_resident_session_needs_no_new_bytes():
    log = []
    srv = _server(budget=50, slots=1)
    S = StubSession("S", 40, last_use=1.0, log=log)
    srv.sessions = {0: S}
    srv.in_use = 40
    slot, admitted = srv._acquire(_req(4), 0, owner=S)
    assert admitted == 0 and srv.in_use == 40 and log == []


def test_owner_waits_for_its_own_eviction_to_finish():
    log = []
    srv = _server(budget=100, slots=1)
    S = StubSession("S", 40, last_use=1.0, log=log)
    S.evicting = True
    srv.sessions = {0: S}
    srv.in_use = 40
    got = []
    t = threading.Thread(target=lambda: got.append(srv._acquire(_req(5), 0, owner=S)))
    t.start()
    time.sleep(0.05)
    assert not got  # still waiting for the copy
    with srv.lock:  # the evicting thread finishes: state spilled, bytes returned
        S.evicting = False
        S.counted = S.resident = False
        srv.in_use -= S.held
        srv.lock.notify_all()
    t.join(5)
    assert got and got[0][1] == 40 and srv.in_use == 40
