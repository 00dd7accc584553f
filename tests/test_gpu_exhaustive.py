"""Exhaustive checks of the fast path's arithmetic on the GPU, through the C ABI.

The binary64 fast path forms RN(j * w[i]) as fma(1 + j 2^-52, b, -b) with
b = 2^52 w[i] and both operands built from bits, and the binary64 batch kernel
also as a correctly rounded product in 32-bit integer arithmetic, both on the
signed entries +-b it keeps; each must equal IEEE multiplication (negated for
the negative entries) for every abscissa j < 2^24 of every layer (5 x 2^31
products).  The bfloat16 outputs round binary32
values with an integer routine that must equal CUDA's RN-even conversion for
every finite binary32 pattern; the modified ziggurat's binary32 and bfloat16
outputs round binary64 values with two more, checked against CUDA's conversions
on 2^32 values each and on 2^31 exact ties or tie neighbours each.  The tail step's table-driven binary64 log must
stay within one ulp of CUDA's log (both are within about an ulp of the exact
value) on 2^31 uniforms spread over (0, 1), and equal it almost always.

The slow tests are decided in binary32 first and in binary64 only inside a
margin meant to cover every binary32 error; on 2^27 inputs per test, half of
them packed within 2^-8 of the test's boundary and the tails' uniforms spread
down to 2^-53, no binary32 decision may differ from the binary64 definition.
"""

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_product_and_bf16_rounding_exhaustive():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_19493_gb300 as Z
    Z.zig_tables_init(0)
    r = Z._binding.zig_selfcheck()
    assert r["products_checked"] == 5 * 128 * 2 ** 24
    # every finite binary32 pattern (to bfloat16); 2^32 binary64 values to binary32 and
    # to bfloat16 each, and 2^31 ties or tie neighbours for each
    assert r["roundings_checked"] == 2 ** 32 - 2 * (2 ** 23) + 6 * 2 ** 31
    assert r["product_mismatches"] == 0
    assert r["rounding_mismatches"] == 0
    assert r["logs_beyond_one_ulp"] == 0
    assert r["logs_not_equal"] < 0.01 * 2 ** 31


def test_binary32_filters_agree_with_binary64_definitions():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_19493_gb300 as Z
    Z.zig_tables_init(0)
    r = Z._binding.zig_filtercheck()
    for name, c in r.items():
        assert c["checked"] == 2 ** 27 or (name == "wedge128" and c["checked"] > 2 ** 26), (name, c)
        assert c["wrong"] == 0, (name, c)
        # the boundary was reached (inputs inside the margin), and the uniform half
        # is nearly all decided in binary32
        assert 0 < c["undecided"] < 0.55 * c["checked"], (name, c)
