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


def test_reference_arm_reports_the_same_workload(monkeypatch, capsys):
    """bench.py --impl reference prints one contract line on the GPU arm's
    workload config (the oracle's timing is stubbed: 0.3 s fixed + 0.1 s per
    pass), with the reference arm's own keys."""
    import argparse

    import numpy as np

    monkeypatch.setattr(bench, "_oracle_solve_seconds", lambda ub, g, m, n: 0.3 + 0.1 * n)
    monkeypatch.setattr(bench, "_fields", lambda seeds: [np.zeros((8, 8), dtype=np.float32) for _ in seeds])
    args = argparse.Namespace(gpus=1, steps=2, warmup=1, impl="reference", method="bicgstab", space="physical",
                              batch=bench.WORKLOAD["batch"])
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["config"] == bench._workload_config(args, 1)
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    n = bench._golden_count("bicgstab", 0) or 160
    assert abs(line["value"] - 2048 * 2048 / (0.3 + n * 0.1) / 1e6) < 1e-9


def test_body_dram_fraction_uses_the_captured_bytes(monkeypatch):
    """roofline_solve reports the body's DRAM-byte rate (ncu bytes per launch
    from profiles/traffic.json) beside its algorithmic rate, only when every
    pass of the body has a capture."""
    class FakeLib:
        @staticmethod
        def time_body(shape, gamma, B, method, reps, space):
            return 2.0                                      # ms
    passes = [{"kind": "xfwd", "op": 3, "bytes": 4e9, "ms": 1.0}, {"kind": "filt", "op": 0, "bytes": 2e9, "ms": 1.0}]
    captured = {("xfwd", 3, "physical"): 3e9, ("filt", 0, "physical"): 1e9}
    monkeypatch.setattr(bench, "_traffic", lambda k, o, sp: captured.get((k, o, sp)))
    ent = bench._solve_entry(FakeLib, passes, (64, 64), 0.1, 1, "bicgstab", "physical", 1000.0, "measured")
    assert abs(ent["achieved"] - 3000.0) < 1e-9 and abs(ent["frac"] - 3.0) < 1e-12
    assert abs(ent["dram"]["bytes_per_body"] - 4e9) < 1e-3 and abs(ent["dram"]["frac"] - 2.0) < 1e-12
    captured.pop(("filt", 0, "physical"))
    assert "dram" not in bench._solve_entry(FakeLib, passes, (64, 64), 0.1, 1, "bicgstab", "physical", 1000.0, "m")


def test_3d_bicgstab_pass_bytes():
    """A 3D BiCGSTAB pass adds the y passes around each filter pass: per G the
    spectrum goes S1 -> S2 (forward y), S2 -> S2 (filter along z), S2 -> S1
    (inverse y); 15 field vectors and 16 spectra per pass (the 31
    vector-equivalents of the design notes, of which a fused yz-plane pass
    would remove 8 spectra)."""
    n, B = 512, 3
    P, SP = n ** 3, (n // 2 + 1) * n * n
    v, s = 4 * P * B, 8 * SP * B
    body = [("xfwd", 3), ("yfwd", 3), ("filt", 0), ("yinv", 0), ("xinv", 6),
            ("xfwd", 4), ("yfwd", 4), ("filt", 2), ("yinv", 2), ("xinv", 7)]
    got = [bench._pass_bytes(k, o, P, SP, B, "bicgstab") for k, o in body]
    assert sum(got) == 15 * v + 16 * s
    assert got[1] == got[2] == got[3] == 2 * s
