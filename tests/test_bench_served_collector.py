"""bench.py's served-trace client against a fake server (CPU only).

A finished result the client has not released stays charged against the
server's memory budget.  A client that waited on its requests strictly in
submission order, releasing each result only after the previous one, could
starve the admission of a large request: while it waited on the large one,
the small requests behind it finished and kept their memory, so the large
one never fit.  The fake server below reproduces that admission rule (arrival
order, small requests may pass a large one waiting for memory, memory held
until release); the trace must complete, with every request served.
"""

import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


class FakeFe:
    FE_STATE_PENDING, FE_STATE_ADMITTED, FE_STATE_RUNNING = 0, 1, 2
    FE_STATE_DONE, FE_STATE_FAILED, FE_STATE_CANCELLED = 3, 4, 5
    FE_DETERMINISTIC = 1

    class FeError(RuntimeError):
        pass

    BUDGET = 8          # memory units
    LARGE_COST = 7      # a large request's units; a small one takes 1

    def __init__(self):
        self.mu = threading.Lock()
        self.cv = threading.Condition(self.mu)
        self.tickets = {}
        self.order = []     # pending ticket ids, arrival order
        self.in_use = 0
        self.next_id = 1
        self.stop = False
        self.admitted = self.completed = 0
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()

    @staticmethod
    def now_us():
        return time.perf_counter() * 1e6

    def _run(self):
        while True:
            with self.cv:
                if self.stop:
                    return
                now = self.now_us()
                for t in self.tickets.values():
                    if t["state"] == self.FE_STATE_RUNNING and now >= t["due"]:
                        t["state"] = self.FE_STATE_DONE
                        t["t_done_us"] = now
                        self.completed += 1
                        self.cv.notify_all()
                blocked = False
                for tid in list(self.order):
                    t = self.tickets[tid]
                    cost = self.LARGE_COST if t["large"] else 1
                    if blocked and t["large"]:
                        continue
                    if self.in_use + cost > self.BUDGET:
                        blocked = True
                        continue
                    self.order.remove(tid)
                    self.in_use += cost
                    t.update(state=self.FE_STATE_RUNNING, cost=cost, t_admit_us=now, t_ready_us=now, t_start_us=now,
                             due=now + (5000.0 if t["large"] else 3000.0))
                    self.admitted += 1
            time.sleep(2e-4)

    # --- the binding's calls used by serve_trace ---
    def fe_server_start(self, ctx, n_streams, max_batch, budget):
        return self

    def make_request(self, key, Dd, n_dofs, k_ref=None, seed=0, mode=1):
        return {"large": Dd == "large"}

    def fe_batch_submit(self, sv, reqs):
        out = []
        with self.cv:
            for r in reqs:
                tid = self.next_id
                self.next_id += 1
                now = self.now_us()
                self.tickets[tid] = dict(state=self.FE_STATE_PENDING, large=r["large"], t_submit_us=now,
                                         t_admit_us=0.0, t_ready_us=0.0, t_start_us=0.0, t_done_us=0.0)
                self.order.append(tid)
                out.append(tid)
        return out

    def _result(self, tid):
        t = self.tickets[tid]
        return {k: t[k] for k in ("state", "t_submit_us", "t_admit_us", "t_ready_us", "t_start_us", "t_done_us")}

    def fe_poll(self, sv, tid):
        with self.cv:
            return self._result(tid)

    def fe_wait(self, sv, tid, timeout):
        end = time.perf_counter() + timeout
        with self.cv:
            while self.tickets[tid]["state"] not in (self.FE_STATE_DONE, self.FE_STATE_FAILED):
                left = end - time.perf_counter()
                if left <= 0:
                    raise self.FeError("timeout")
                self.cv.wait(left)
            return self._result(tid)

    def fe_release(self, sv, tid):
        with self.cv:
            t = self.tickets.pop(tid)
            self.in_use -= t.get("cost", 0)

    def fe_server_stats_get(self, sv):
        with self.cv:
            st = dict.fromkeys(("launches", "batched_requests", "patterns_built", "evictions", "rebuilds",
                                "admission_waits", "peak_bytes_in_use", "budget_bytes", "n_pending", "n_to_build",
                                "n_ready", "n_big_jobs", "n_running", "n_inflight_groups", "failed",
                                "cached_patterns"), 0)
            st.update(submitted=self.next_id - 1, admitted=self.admitted, completed=self.completed,
                      bytes_in_use=self.in_use, alloc_ms_max=0.0, alloc_ms_total=0.0)
            return st

    def fe_server_timeline(self, sv):
        return []

    def fe_server_stop(self, sv):
        with self.cv:
            self.stop = True
        self.th.join()


class FakeTraffic:
    def __init__(self, fe):
        self.fe = fe
        self.np = np
        self.classes = {(8, 1): ("small", None, 729, 512 * 64), (128, 3): ("large", None, 3 * 129 ** 3, 10 ** 9)}


def test_served_trace_releases_results_out_of_order(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "SERVE_WAIT_S", 10.0)
    fe = FakeFe()
    traffic = FakeTraffic(fe)
    m = 300
    arrivals = np.arange(m) * 0.5e-3  # one request per 0.5 ms, each small one runs 3 ms
    # a large cold request every 25: small requests fill the memory the large
    # one needs while the trace lasts; once it ends, the large ones fit only if
    # the finished small ones behind them are released
    kinds = [((128, 3), True, False) if k % 25 == 10 else ((8, 1), False, True) for k in range(m)]
    t0 = time.perf_counter()
    out = bench.serve_trace(None, traffic, arrivals, kinds, 4, 64)
    assert time.perf_counter() - t0 < 30
    assert out["completed"] == m and out["requests"] == m
    assert fe.in_use == 0  # every result was released
