"""Write the oracle's stored tables (``oracle/tables/*.txt``) from ``oracle.tables``.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  This script calls only
``oracle/`` code.  The GPU machine has no mpmath, so the oracle reads the stored
text there; ``tests/test_oracle_tables.py`` re-runs the construction where mpmath
exists and checks the stored files byte for byte.

    python -m oracle.gen_tables          # rewrite both files
"""

from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "tables")


def render_zig128(t) -> str:
    lines = [
        "# oracle zig128 tables: 128-level original ziggurat (Marsaglia-Tsang geometry,",
        "# base layer = R f(R) + f(R)/R).  Written by oracle/gen_tables.py; do not edit.",
        "# columns: i k[i] w[i] y[i]   (w, y as C99 hex floats)",
        f"R {t['R'].hex()}",
        f"v {t['v'].hex()}",
    ]
    for i in range(128):
        lines.append(f"{i} {t['k'][i]} {t['w'][i].hex()} {t['y'][i].hex()}")
    return "\n".join(lines) + "\n"


def render_zig256(t) -> str:
    lines = [
        "# oracle zig256 tables: 256-slot modified ziggurat (equal-area inscribed rectangles,",
        "# alias-selected overhangs and tail).  Written by oracle/gen_tables.py; do not edit.",
        f"n_r {t['n_r']}",
        f"x0 {t['x0'].hex()}",
        "# fast: j xs[j]",
    ]
    for j in range(t["n_r"]):
        lines.append(f"xs {j} {t['xs'][j].hex()}")
    lines.append("# overhang: r ox odx oy ody kind qa")
    for r in range(1, t["n_r"] + 1):
        lines.append(f"oh {r} {t['ox'][r].hex()} {t['odx'][r].hex()} {t['oy'][r].hex()} "
                     f"{t['ody'][r].hex()} {t['kind'][r]} {t['qa'][r]}")
    lines.append("# alias: b thr alias")
    for b in range(256):
        lines.append(f"al {b} {t['thr'][b]} {t['alias'][b]}")
    return "\n".join(lines) + "\n"


def main(argv=None) -> int:
    sys.path.insert(0, os.path.dirname(HERE))
    from oracle import tables
    os.makedirs(OUT_DIR, exist_ok=True)
    with open(os.path.join(OUT_DIR, "zig128.txt"), "w") as fh:
        fh.write(render_zig128(tables.zig128_tables()))
    with open(os.path.join(OUT_DIR, "zig256.txt"), "w") as fh:
        fh.write(render_zig256(tables.zig256_tables()))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
