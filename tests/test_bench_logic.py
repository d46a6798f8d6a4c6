"""Host logic of bench.py that needs no GPU: the serving driver's accounting against a fake server
(every request answered, latency and queueing counted from the scheduled arrival, the host-memory
hold-back respected), the roofline arithmetic, and the committed ncu traffic record matching the
current source of the kernel it describes."""
import json
import os
import threading
import time

import numpy as np

import bench


class FakeServer:
    """Serves each request after a fixed delay per right-hand side, one at a time, in arrival
    order; records the host bytes it holds (b and x of every unfinished request)."""

    def __init__(self, per_rhs_s):
        self.per_rhs_s = per_rhs_s
        self.lock = threading.Lock()
        self.reqs = {}
        self.next_id = 0
        self.busy_until = 0.0
        self.held = 0
        self.max_held = 0

    def submit(self, hid, b, n, tol):
        assert b.flags["C_CONTIGUOUS"] and b.shape[0] == n
        with self.lock:
            rid = self.next_id
            self.next_id += 1
            now = time.perf_counter()
            start = max(now, self.busy_until)
            done = start + self.per_rhs_s * n
            self.busy_until = done
            self.reqs[rid] = (now, start, done, b.copy(), n)
            self.held += 2 * b.nbytes
            self.max_held = max(self.max_held, self.held)
        return rid

    def wait(self, rid, x, n):
        t_sub, start, done, b, _ = self.reqs[rid]
        d = done - time.perf_counter()
        if d > 0:
            time.sleep(d)
        x[...] = 2.0 * b
        with self.lock:
            self.held -= 2 * b.nbytes
            del self.reqs[rid]
        st = [{"iterations": 15, "cycles": 2, "converged": True, "true_residual": 5e-11} for _ in range(n)]
        return st, (start - t_sub, done - t_sub, done - start), 0


def test_serving_run_accounts_from_the_scheduled_arrival_and_holds_back_within_budget(monkeypatch):
    pools = [np.ones((12, 4, 12), dtype=np.complex128), np.ones((12, 6, 12), dtype=np.complex128)]
    one_rhs = pools[1][0].nbytes
    # a budget of 30 right-hand sides' bytes (the b and x copies of one 12-RHS request take 24):
    # the driver must hold requests back
    monkeypatch.setattr(bench, "SERVING_HOST_BUDGET", 30 * one_rhs)
    srv = FakeServer(per_rhs_s=0.002)
    rng = np.random.default_rng(7)
    rec = bench.serving_run(None, srv, [0, 1], pools, 400.0, 40, rng)
    assert rec["requests"] == 40
    assert rec["all_converged"]
    assert srv.max_held <= 30 * one_rhs
    # every latency covers at least the request's own service time
    assert rec["p50_latency_s"] >= 0.002
    # the offered load (400 req/s of 1-12 RHS) is far above the 500 RHS/s of the fake server,
    # so queueing grows from the first quarter to the last
    assert rec["queue_s_last_quarter"] > rec["queue_s_first_quarter"]
    assert rec["rhs"] >= 40


def test_roofline_picks_the_binding_roof(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: (6778.7, "measured"))
    kernel = os.path.join(bench.ROOT, "paper_1307_6101_gb300", "csrc", "fine.cu")
    # 10 launches of 0.042 ms and 52.7 MB each; 743 MFLOP per launch: 14 FLOP/B, above the ridge
    prof = (0.42, 10, 527e6, 32.0)
    r = bench.roofline(prof, 2, kernel, 743.44e6, "three_level_16c32")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 743.44e6 / 0.042e-3 / 1e12) < 0.01
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    assert abs(r["hbm"]["achieved"] - 52.7e6 / 0.042e-3 / 1e9) < 1.0
    # without FLOPs the HBM roof is the entry
    r2 = bench.roofline(prof, 2, kernel, None, "three_level_16c32")
    assert r2["bound"] == "hbm" and r2["unit"] == "GB/s"


def test_committed_traffic_record_matches_the_kernel_source():
    """profiles/fine_sap_sweep_traffic.json was captured from the current source of the fine SAP
    sweep: a change to the kernel needs a new capture (the bench reports null until then)."""
    kernel = os.path.join(bench.ROOT, "paper_1307_6101_gb300", "csrc", "fine.cu")
    with open(os.path.join(bench.ROOT, "profiles", "fine_sap_sweep_traffic.json")) as f:
        d = json.load(f)
    assert d["source_sha256"] == bench.kernel_sha(kernel)
    for key in ("three_level_16c32", "batched_32c64"):
        t = bench.ncu_traffic(kernel, key)
        assert t is not None and t > 0
        # DRAM traffic of a sweep stays at or below its algorithmic bytes (nothing re-read)
        cap = d["captures"][key]
        alg = cap.get("algorithmic_bytes_per_launch", cap.get("algorithmic_bytes_per_launch_captured"))
        got = cap.get("dram_bytes_per_launch_captured", cap["dram_bytes_per_launch"])
        assert got <= alg
