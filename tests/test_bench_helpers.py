"""bench.py's host-side helpers (no GPU): the ALU roofline arithmetic of the
headline kernel and the oracle comparison of sampled output lines."""
import numpy as np

from conftest import ROOT  # noqa: F401  (puts the repository root on sys.path)
import synth


def test_alu_roofline_arithmetic():
    import bench
    L, Nz, C, d = 1080, 513, 25, 5
    r = {"points": 3 * 512 * 512 * Nz, "seconds_per_call_mean": 2e-3}
    out = bench._deriv_alu_roofline(r, {"sm_mhz": 2000.0}, L=L, Nz=Nz, C=C, d=d)
    pair = 3 * 5 * L * np.log2(L) + 2 * 6 * L + 2 * 2 * C * d * 2 + 2 * 2 * Nz
    pairs = 3 * 512 * 512 / 2
    assert abs(out["flops_per_line_pair"] - pair) < 1e-6
    assert abs(out["achieved"] - pair * pairs / 2e-3 / 1e12) < 1e-9
    assert abs(out["peak"] - 152 * 128 * 2 * 2000e6 / 1e12) < 1e-9
    assert abs(out["frac"] - out["achieved"] / out["peak"]) < 1e-12
    assert out["bound"] == "alu" and out["unit"] == "TFLOP/s"
    # no clock sample: the maximum SM clock
    assert abs(bench._deriv_alu_roofline(r, None)["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9


def test_oracle_accuracy_of_sampled_lines():
    import bench
    from oracle import fc, fc_tables
    Mr = fc_tables.fc_matrix(5, 25, table_dir=ROOT + "/tests/golden")
    f = synth.SeparableField(4, 4, 129, rank=2).field(0).reshape(129, -1)
    d1 = fc.fc_deriv_z(f, 1.0, Mr, 1, axis=0)
    d2 = fc.fc_deriv_z(f, 1.0, Mr, 2, axis=0)
    r = {"_samples": (f, d1 * (1 + 3e-6), d2)}
    bench.oracle_accuracy(r)
    assert "_samples" not in r
    assert abs(r["rel_l2_err_d1_vs_oracle"] - 3e-6) < 1e-12
    assert r["rel_l2_err_d2_vs_oracle"] == 0.0
    r = {}
    bench.oracle_accuracy(r)          # nothing sampled: nothing reported
    assert r == {}
