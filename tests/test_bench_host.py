"""Host logic of bench.py that needs no GPU: the served end-to-end line counts a
request only when it succeeded with the stored radius, warms one request per
large worker outside the timed region, and closes the server."""
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _FakeServer:
    log = []

    def __init__(self, budget_bytes, **kw):
        self.n = 0
        self.closed = False
        _FakeServer.log.append(self)

    def submit(self, C, R, active_cap=None):
        self.n += 1
        return self.n

    def wait(self, t):
        # every third request fails; the others return radius 1
        return {"rc": -3 if t % 3 == 0 else 0, "r": 1.0, "latency_s": 0.001 * t}

    def close(self):
        self.closed = True


class _FakeMeb:
    Server = _FakeServer


def test_served_e2e_counts_only_correct_requests():
    pC = torch.zeros(16, 4, dtype=torch.float64)
    pR = torch.zeros(16, dtype=torch.float64)
    out = bench.served_e2e(_FakeMeb, pC, pR, 1.0, 9)
    sv = _FakeServer.log[-1]
    assert sv.closed and sv.n == 2 + 9
    # tickets 3..11 are timed; 3, 6 and 9 fail
    assert out["requests"] == 9 and out["ok"] == 6
    assert out["value"] == out["ok"] / out["wall_s"]
    assert out["h2d_bytes_per_step"] == 16 * 4 * 8 + 16 * 8
    assert out["max_latency_ms"] == 11.0
    # a radius off the stored one counts as a failure
    assert bench.served_e2e(_FakeMeb, pC, pR, 2.0, 4)["ok"] == 0
