"""Output quality per dtype on the GPU: 2^26 variates from 2^16 streams.

The binary64 outputs match the oracle element by element (test_gpu_parity.py);
here the binary32 and bfloat16 outputs of the same streams are held within one
step of the binary64 ones rounded to nearest, and every type passes a KS test against Phi
(bfloat16: against the exactly rounded normal), with the mass beyond |x| > 3
within 6 standard deviations of its expectation.
"""

import numpy as np
import pytest

from paper_2405_19493_gb300 import quality as Q
from paper_2405_19493_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytest.importorskip("scipy")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def outputs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_19493_gb300 as Z
    Z.zig_tables_init(0)
    n_s, L = 1 << 16, 1024
    sd = torch.from_numpy(W.seeds(n_s, base=0xC0FFEE).view(np.int64)).cuda()
    res = {}
    for dt, tdt in (("f64", torch.float64), ("f32", torch.float32), ("bf16", torch.bfloat16)):
        o = torch.empty(n_s * L, dtype=tdt, device="cuda")
        Z.zig_generate("l64x128mix", "zig128", sd, o, uniform_len=L, dtype=dt)
        res[dt] = o
    torch.cuda.synchronize()
    assert Z.zig_device_status(0) == 0
    return res


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_ks_and_tail(outputs, dt):
    x = outputs[dt]
    if dt == "bf16":
        r = Q.ks_bf16_exact(torch, x)
        assert r["p_value"] > 1e-6, r
        assert r["D_vs_phi"] < 2e-3, r          # the rounding floor, not a defect
    else:
        r = Q.ks_grid(torch, x, K=1 << 16)
        assert r["p_value"] > 1e-6, r
    t = Q.tail_mass(torch, x, dt)
    assert abs(t["z_score"]) < 6, t


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_narrow_outputs_within_one_ulp_of_f64(outputs, dt):
    # within one step of RN(z64), hence within 1.5 ulp of z64 itself
    e = Q.error_vs_f64(torch, outputs[dt], outputs["f64"], dt)
    assert e["max_steps_from_nearest"] <= 1, e
    assert e["max_err_ulp"] <= 1.5, e
    assert e["max_rel_err"] <= 1.5 * 2.0 ** (1 - Q.MANT_BITS[dt]), e
