"""The benchmark's byte accounting (no GPU): the algorithmic bytes of one
BiCGSTAB pass (Algorithm 4) counted vector by vector from the algorithm, and
the rule that ncu traffic is reported only for the kernel sources it was
measured on."""

import json

import bench


def test_bicgstab_pass_bytes_match_the_algorithm():
    P, B = 2048 * 2048, 16
    SP = (2048 // 2 + 1) * 2048
    v, s = 4 * P * B, 8 * SP * B
    # one BiCGSTAB body in physical space, the launches in order (kind, op)
    body = [("xfwd", 3), ("filt", 0), ("xinv", 6), ("xfwd", 4), ("filt", 2), ("xinv", 7)]
    got = [bench._pass_bytes(k, o, P, SP, B, "bicgstab") for k, o in body]
    expected = [
        v * (3 + 1) + s,   # p = r + beta (p - omega q): reads r, p, q; writes p; spectrum out
        2 * s,             # filter: spectrum in and out
        s + v * (1 + 1),   # q = G p: spectrum in; reads f0 for (f0, q), writes q
        v * (2 + 1) + s,   # s = r - alpha q: reads r, q; writes s; spectrum out
        2 * s,             # filter with the (s, s), (s, Gs), (Gs, Gs) Parseval dots
        s + v * (4 + 2),   # t = G s; u += alpha p + omega s; r = s - omega t: reads p, s, u, f0; writes u, r
    ]
    assert got == expected
    # 15 field vectors and 8 spectra: the 23 vector-equivalents per pass of the design notes
    assert sum(got) == 15 * v + 8 * s


def test_traffic_is_reported_only_for_the_measured_kernels(tmp_path, monkeypatch):
    rec = {"kernel_sha": "abc", "bytes_per_launch": {"physical:xinv:7": 123.0}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_sha", lambda: "abc")
    assert bench._traffic("xinv", 7, "physical") == 123.0
    assert bench._traffic("xinv", 6, "physical") is None
    monkeypatch.setattr(bench, "_kernel_sha", lambda: "changed")
    assert bench._traffic("xinv", 7, "physical") is None


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_mpoints(1, 16, 2048 * 2048, 0.5) * 4 == bench.whole_job_mpoints(4, 16, 2048 * 2048, 0.5)
