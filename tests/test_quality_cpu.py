"""The distribution checks used to report output quality, on CPU tensors with known answers."""

import numpy as np
import pytest

from paper_2405_19493_gb300 import quality as Q

torch = pytest.importorskip("torch")
pytest.importorskip("scipy")


def normals(n, seed=1):
    return torch.from_numpy(np.random.default_rng(seed).standard_normal(n))


def test_ks_grid_accepts_normal_and_rejects_shift():
    x = normals(1 << 20)
    r = Q.ks_grid(torch, x, K=1 << 12, chunk=1 << 18)
    assert r["p_value"] > 1e-4 and r["D"] < 3 / np.sqrt(x.numel())
    bad = Q.ks_grid(torch, x + 0.01, K=1 << 12, chunk=1 << 18)
    # a shift of 0.01 moves the CDF by about 0.01 * phi(0) = 0.004
    assert bad["D"] > 0.003 and bad["p_value"] < 1e-10


def test_ks_bf16_exact_sees_rounding_but_not_as_an_error():
    x = normals(1 << 20, seed=2)
    xb = x.float().to(torch.bfloat16)            # RN to binary32, then RN to bfloat16
    r = Q.ks_bf16_exact(torch, xb, chunk=1 << 18)
    assert r["p_value"] > 1e-4
    assert r["D_vs_phi"] > 5e-4                  # the rounding floor against Phi itself
    # truncation toward zero instead of rounding moves the CDF by about half a
    # spacing times the density (~1e-3 near |x| = 1): visible at n = 2^24
    x = normals(1 << 24, seed=5)
    tr = (x.float().view(torch.int32) & ~0xFFFF).view(torch.float32).to(torch.bfloat16)
    assert Q.ks_bf16_exact(torch, tr, chunk=1 << 22)["p_value"] < 1e-8


def test_tail_mass_expectations():
    assert Q.tail_mass(torch, torch.zeros(4), "f64")["expected"] == pytest.approx(0.0026997960632601866, rel=1e-12)
    # bfloat16 spacing at 3 is 2^-6: RN(z) > 3 needs z > 3 + 2^-7
    from scipy.special import ndtr
    assert Q.tail_mass(torch, torch.zeros(4), "bf16")["expected"] == pytest.approx(2 * ndtr(-(3 + 2 ** -7)))
    x = normals(1 << 20, seed=3)
    r = Q.tail_mass(torch, x, "f64", chunk=1 << 18)
    assert abs(r["z_score"]) < 5
    assert Q.tail_mass(torch, x * 1.05, "f64", chunk=1 << 18)["z_score"] > 10


def test_error_vs_f64_in_ulps():
    z = normals(1 << 16, seed=4)
    e = Q.error_vs_f64(torch, z.float(), z, "f32", chunk=1 << 14)
    assert e["max_err_ulp"] <= 0.5 and e["outputs_not_nearest"] == 0 and e["max_steps_from_nearest"] == 0
    assert e["max_rel_err"] <= 2.0 ** -24
    # one ulp off everywhere: reported as 1 ulp, every output not nearest
    up = torch.from_numpy(np.nextafter(z.float().numpy(), np.float32(np.inf)))
    e2 = Q.error_vs_f64(torch, up, z, "f32", chunk=1 << 14)
    assert 0.5 < e2["max_err_ulp"] <= 1.5 and e2["outputs_not_nearest"] == z.numel()
    assert e2["max_steps_from_nearest"] == 1
    # binary64 -> binary32 -> bfloat16 rounds twice: a few outputs are a step off
    eb = Q.error_vs_f64(torch, z.float().to(torch.bfloat16), z, "bf16", chunk=1 << 14)
    assert eb["max_err_ulp"] <= 0.5 + 2.0 ** -15 and eb["max_steps_from_nearest"] <= 1


def test_round_to_precision_is_one_rounding():
    # RN to 8 bits of 1 + 2^-8 + 2^-30: above the midpoint, so it rounds up, where
    # rounding first to binary32 (1 + 2^-8, a tie) and then to even gives 1
    z = torch.tensor([1 + 2.0 ** -8 + 2.0 ** -30, -(1 + 2.0 ** -8 + 2.0 ** -30), 1 + 2.0 ** -8,
                      1 + 3 * 2.0 ** -8, 2.5], dtype=torch.float64)
    got = Q.round_to_precision(torch, z, 8).tolist()
    assert got == [1 + 2.0 ** -7, -(1 + 2.0 ** -7), 1.0, 1 + 4 * 2.0 ** -8, 2.5]
    assert z.float().to(torch.bfloat16)[0].item() == 1.0


def test_serial_chi2_sees_dependence_within_streams():
    x = normals(1 << 20, seed=6)
    r = Q.serial_chi2(torch, x, stream_len=1 << 10, lag=1)
    assert r["p_value"] > 1e-4 and r["pairs"] == (1 << 10) * ((1 << 10) - 1)
    # an AR(1) sequence with correlation 0.05 is flagged
    a = np.empty(1 << 20)
    z = np.random.default_rng(7).standard_normal(1 << 20)
    a[0] = z[0]
    for t in range(1, len(a)):
        a[t] = 0.05 * a[t - 1] + np.sqrt(1 - 0.05 ** 2) * z[t]
    assert Q.serial_chi2(torch, torch.from_numpy(a), stream_len=1 << 10, lag=1)["p_value"] < 1e-10
