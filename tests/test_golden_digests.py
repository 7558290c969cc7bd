"""The stored full-size digests (tests/golden/full_size_digests.json) are the
oracle's: recomputed here from ``oracle/`` for the workloads small enough to
rerun in seconds (lines_2d and the smallest batched scenes), and checked for
shape and consistency everywhere else. The file is written by
tests/golden/make_full_size_digests.py, which calls only the oracle."""
import hashlib
import json
import os

import numpy as np

import oracle
from paper_1503_06029_gb300 import inputs

DIGESTS = os.path.join(os.path.dirname(__file__), "golden", "full_size_digests.json")


def _load():
    with open(DIGESTS) as f:
        return json.load(f)


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def test_digest_file_covers_the_workloads():
    g = _load()
    spec = inputs.scene_batch_spec()
    assert len(g["batch_scenes"]) == len(spec.n) == 1024
    for i, e in enumerate(g["batch_scenes"]):
        assert e["scene"] == i and e["n"] == int(spec.n[i]) and e["ell"] == int(spec.ell[i])
        assert 0 < e["n_cells"] <= e["n"] and 0 <= e["n_edges"] <= e["n_cells"] * e["ell"] // 2
    ch = g["chains"]
    assert (ch["n"], ch["ell"], ch["n_cells"], ch["n_edges"]) == (5 * 2**20, 1024, 4190741, 3932003)
    assert g["planes_3d"]["n"] == 2**24 and g["planes_3d"]["n_cells"] <= 43745
    sp = g["spheres_3d"]
    assert (sp["n"], sp["ell"]) == (2**24, 64) and 0 < sp["n_edges"] <= sp["n_cells"] * 32


def test_digests_match_the_oracle_on_small_workloads():
    g = _load()
    sc = inputs.lines_2d()
    c, e = oracle.build(sc.pts, sc.a, sc.b, 32)
    assert (_sha(c), _sha(e)) == (g["lines_2d"]["cells_sha256"], g["lines_2d"]["edges_sha256"])
    spec = inputs.scene_batch_spec()
    small = sorted(range(len(spec.n)), key=lambda s: int(spec.n[s]))[:6]
    for s in small:
        sc = inputs.batch_scene(spec, s)
        c, e = oracle.build(sc.pts, sc.a, sc.b, 64)
        want = g["batch_scenes"][s]
        assert (len(c), len(e)) == (want["n_cells"], want["n_edges"])
        assert (_sha(c), _sha(e)) == (want["cells_sha256"], want["edges_sha256"])
