"""The library's generated tables equal the oracle's, bit for bit (CPU only).

The two sides are built independently: the oracle with mpmath at 50 digits
(bisection, ternary search), the library with the standard ``decimal`` module at
80 digits (regula falsi, safeguarded Newton).  Each rounds once to binary64, so
agreement of every entry checks both constructions against each other.
"""

import os
import re

import numpy as np
import pytest

import oracle as O

INC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2405_19493_gb300", "csrc", "zig_tables.inc")


def _parse_inc():
    txt = open(INC).read()
    scal = dict(re.findall(r"static const \w+ (\w+) = ([^;]+);", txt))
    arrs = {}
    for name, body in re.findall(r"static const \w+ (\w+)\[\d+\] = \{([^}]*)\};", txt):
        vals = [v.strip() for v in body.replace("\n", " ").split(",") if v.strip()]
        arrs[name] = vals
    return scal, arrs


def _num(tok):
    tok = tok.rstrip("uUlLf") if not tok.startswith("0x") else tok
    if tok.startswith("0x") or tok.startswith("-0x"):
        if "p" in tok:
            return float.fromhex(tok.rstrip("f"))
        return int(tok.rstrip("uUlL"), 16)
    return int(tok.rstrip("uUlL"))


def test_zig128_tables_identical():
    scal, arrs = _parse_inc()
    t = O.read_zig128()
    assert _num(scal["ZIG128_R"]) == t["R"]
    assert _num(scal["ZIG128_V"]) == t["v"]
    assert [_num(v) for v in arrs["ZIG128_K"]] == t["k"]
    assert [_num(v) for v in arrs["ZIG128_W"]] == t["w"]
    assert [_num(v) for v in arrs["ZIG128_Y"]] == t["y"]
    # the binary32 copy is the once-rounded abscissa: within half an ulp32 of w
    w32 = np.array([float.fromhex(v.rstrip("f")) for v in arrs["ZIG128_W32"]])
    w = np.array(t["w"])
    assert np.all(np.abs(w32 - w) <= np.spacing(w32.astype(np.float32)).astype(np.float64) / 2)
    assert np.array_equal(w32.astype(np.float32).astype(np.float64), w32)


def test_zig256_tables_identical():
    scal, arrs = _parse_inc()
    t = O.read_zig256()
    n = t["n_r"]
    assert int(scal["ZIG256_NR"]) == n
    assert _num(scal["ZIG256_X0"]) == t["x0"]
    assert [_num(v) for v in arrs["ZIG256_XS"]] == t["xs"]
    for lib, orc in (("OX", "ox"), ("ODX", "odx"), ("OY", "oy"), ("ODY", "ody")):
        assert [_num(v) for v in arrs["ZIG256_" + lib]] == t[orc][1:], lib
    assert [int(v) for v in arrs["ZIG256_KIND"]] == t["kind"][1:]
    assert [_num(v) for v in arrs["ZIG256_QA"]] == t["qa"][1:]
    assert [_num(v) for v in arrs["ZIG256_THR"]] == t["thr"]
    assert [int(v) for v in arrs["ZIG256_ALIAS"]] == t["alias"]


def test_generated_file_is_current():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "gen_tables", os.path.join(os.path.dirname(INC), "gen_tables.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert open(INC).read() == mod.render()


def test_c_abi_tables_equal_the_oracle():
    """zig_tables_get through the C ABI (no device needed) against the oracle's tables."""
    import paper_2405_19493_gb300 as Z
    t = Z.zig_tables_get("zig128")
    o = O.read_zig128()
    assert t["R"] == o["R"] and t["V"] == o["v"]
    assert t["k"] == o["k"] and t["w"] == o["w"] and t["y"] == o["y"]
    u = Z.zig_tables_get("zig256")
    o = O.read_zig256()
    n = o["n_r"]
    assert u["n_r"] == n and u["x0"] == o["x0"]
    assert u["xs"][:n] == o["xs"] and all(v == 0.0 for v in u["xs"][n:])
    for name in ("ox", "odx", "oy", "ody", "qa"):
        assert u[name][1:n + 1] == o[name][1:], name
    assert u["kind"][1:n + 1] == o["kind"][1:]
    assert u["thr"] == o["thr"] and u["alias"] == o["alias"]
    assert Z.zig_tables_get("polar") == {}
