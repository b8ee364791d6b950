"""Writes the stored expected values under tests/golden/.

closed_forms.json: values that follow from closed forms alone (no oracle, no
CUDA path), each with its derivation:
  * triangles of K_n = C(n,3); of the wheel W_k (hub + k-cycle, k >= 4) = k;
    of the 4-neighbour grid = 0 (bipartite).
  * PageRank (GAP form, Alg. 4) on the star K_{1,s}: with a = (1-alpha)/n,
    n = s+1, the centre gets alpha*r_l from each leaf (leaf degree 1) and each
    leaf gets alpha*r_c/s, so r_c = a + alpha*s*r_l and r_l = a + alpha*r_c/s,
    giving r_c = a(1 + alpha*s)/(1 - alpha^2).

rmat12_oracle.json: the oracle's results on the seeded R-MAT scale-12 graph
(edge factor 16, seed 20210404), written by calling only ``gen`` and
``oracle``.

rmat22_oracle.json: the oracle's results on the benchmark graph, R-MAT scale
22 (edge factor 16, seed 20210404): the triangle count of Alg. 6 as written
(method AUTO; several minutes on one core) and, for each of the 16 seeded BFS
sources, the depth and level histogram of Alg. 1.  Written by calling only
``gen`` and ``oracle``.

Run from the repository root:  python tests/golden/make_golden.py [--skip-rmat22]
"""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gen      # noqa: E402
import oracle   # noqa: E402


def closed_forms():
    tri = [{"graph": "complete", "args": [n], "t": math.comb(n, 3), "why": "C(n,3)"} for n in (3, 10, 40)]
    tri += [{"graph": "wheel", "args": [k], "t": k, "why": "one triangle per rim edge"} for k in (4, 9, 100)]
    tri += [{"graph": "grid", "args": [r, c], "t": 0, "why": "bipartite"} for r, c in ((5, 7), (64, 64))]
    star = []
    for s, alpha in ((5, 0.85), (40, 0.85), (7, 0.5)):
        n = s + 1
        a = (1 - alpha) / n
        rc = a * (1 + alpha * s) / (1 - alpha ** 2)
        rl = a + alpha * rc / s
        star.append({"s": s, "alpha": alpha, "r_centre": rc, "r_leaf": rl})
    return {
        "triangles": {"source": "closed forms (Alg. 6 counts unique 3-cliques, Sec. IV-E)", "cases": tri},
        "pagerank_star": {"source": "fixed point of Alg. 4 (Sec. IV-C) on K_{1,s}, solved by hand",
                          "cases": star},
    }


def rmat12():
    g = gen.rmat(12, 16)
    level, _, depth = oracle.bfs(g, 0)
    return {
        "graph": "R-MAT scale 12, edge factor 16, a/b/c = .57/.19/.19, seed 20210404, symmetrised, deduplicated",
        "nnz": g.nnz,
        "colidx_hash": int(np.bitwise_xor.reduce(g.colidx.astype(np.int64) * 2654435761 % 2**32)),
        "triangles": oracle.tc(g),
        "bfs0_depth": depth,
        "bfs0_level_histogram": np.bincount(level[level >= 0]).tolist(),
    }


def rmat22():
    seed = 20210404
    g = gen.rmat(22, 16, seed=seed)
    srcs = [int(s) for s in gen.sources(g, 16, seed=seed)]
    bfs = []
    for s in srcs:
        level, _, depth = oracle.bfs(g, s)
        bfs.append({"source": s, "depth": depth, "level_histogram": np.bincount(level[level >= 0]).tolist()})
    return {
        "graph": "R-MAT scale 22, edge factor 16, a/b/c = .57/.19/.19, seed 20210404, symmetrised, deduplicated",
        "nnz": g.nnz,
        "triangles": oracle.tc(g, oracle.TC_AUTO),
        "sources": srcs,
        "bfs": bfs,
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "closed_forms.json"), "w") as f:
        json.dump(closed_forms(), f, indent=1)
    with open(os.path.join(HERE, "rmat12_oracle.json"), "w") as f:
        json.dump(rmat12(), f, indent=1)
    if "--skip-rmat22" not in sys.argv:
        with open(os.path.join(HERE, "rmat22_oracle.json"), "w") as f:
            json.dump(rmat22(), f, indent=1)
