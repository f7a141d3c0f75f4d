"""bench.py's host-side helpers (no GPU): the ALU roofline arithmetic of the
headline kernel and the oracle comparison of sampled output lines."""
import numpy as np

from conftest import ROOT  # noqa: F401  (puts the repository root on sys.path)
import synth


def test_alu_roofline_arithmetic():
    import bench
    L, Nz, C, d = 1080, 513, 25, 5
    r = {"points": 3 * 512 * 512 * Nz, "seconds_per_call_mean": 2e-3}
    out = bench._deriv_alu_roofline(r, 78.4, "measured", L=L, Nz=Nz, C=C, d=d)
    pair = 3 * 5 * L * np.log2(L) + 2 * 6 * L + 2 * 2 * C * d * 2 + 2 * 2 * Nz
    pairs = 3 * 512 * 512 / 2
    assert abs(out["flops_per_line_pair"] - pair) < 1e-6
    assert abs(out["achieved"] - pair * pairs / 2e-3 / 1e12) < 1e-9
    assert out["peak"] == 78.4 and out["peak_kind"] == "measured"
    assert abs(out["frac"] - out["achieved"] / out["peak"]) < 1e-12
    assert out["bound"] == "alu" and out["unit"] == "TFLOP/s"


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


def test_band_limited_restriction_and_rk_accuracy_plumbing():
    """bench.band_limited_fields on a 128^2 grid restricted to every 2nd point
    is the same field on 64^2 (the exact-restriction argument of the full-size
    RK error sample), and rk_accuracy reports ~0 for the oracle's own step."""
    import bench
    from oracle import ns
    f128 = bench.band_limited_fields(128, 17, seed=5)
    f64 = bench.band_limited_fields(64, 17, seed=5)
    assert np.abs(f128[:, :, ::2, ::2] - f64).max() < 1e-13
    kw = dict(nu=3.162e-4, kappa=3.162e-4, gamma=1.0)
    P = ns.Params(64, 64, 17, nfields=4, **kw)
    st, _ = ns.rk_step(ns.to_spectral(f64, P), np.zeros((2, 2, 64, P.Kx), complex), P, 1e-3)
    out = np.stack([ns.to_physical(c, P) for c in st])
    res = {"_err_sample": {"Nz": 17, "dt": 1e-3, "seed": 5, "kw": kw, "out": out}}
    bench.rk_accuracy(res)
    assert max(res["rel_l2_err_vs_oracle_per_field"]) < 1e-14 and "_err_sample" not in res
