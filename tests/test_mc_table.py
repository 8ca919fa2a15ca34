"""The library's marching-cubes case table (generated geometrically by
csrc/gen_mc_table.py) equals the oracle's on-the-fly face walk for all 256
cases, in triangle and corner order, and the committed header is what the
generator writes."""
import importlib.util
import os

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2408_05462_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_mc_table", os.path.join(CSRC, "gen_mc_table.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_table_matches_oracle_face_walk():
    gen = _gen()
    table = gen.build_table()
    for caseb in range(256):
        word = table[caseb]
        nt = word >> 60
        tris = [[(word >> (12 * t + 4 * c)) & 15 for c in range(3)] for t in range(nt)]
        ref = oracle.cell_triangles(caseb).tolist()
        assert tris == ref, (caseb, tris, ref)
    # complementary cases cross the same edges
    for caseb in range(256):
        a = set(np.ravel(oracle.cell_triangles(caseb)).tolist())
        b = set(np.ravel(oracle.cell_triangles(255 - caseb)).tolist())
        assert a == b


def test_committed_header_is_generated():
    gen = _gen()
    with open(os.path.join(CSRC, "mc_table.h")) as fh:
        assert fh.read() == gen.render(gen.build_table())
