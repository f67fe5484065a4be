"""Writes kron27_ef32_sources.txt: the 16 seeded sources of the Kronecker
scale-27 workload, drawn from its giant component as the oracle's union-find
finds it.

The workload takes its sources from the giant component (16 seeded random
vertices there, as the paper averages over random sources, Sec. 5.2).
Finding that component needs the whole graph, so it is done once here, with
the oracle only, and stored.  Needs about 80 GB of host memory and several
minutes (generation, then a single-threaded union-find over 8.6e9 edges):

    python tests/golden/make_kron27_sources.py [output path]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

SCALE, EF, GEN_SEED, SRC_SEED, COUNT = 27, 32, 1, 2, 16
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kron27_ef32_sources.txt")


def main(out=OUT):
    t0 = time.time()
    g = gg.kronecker(SCALE, EF, seed=GEN_SEED)
    t1 = time.time()
    lab = oracle.cc_g(g)
    t2 = time.time()
    roots, sizes = np.unique(lab, return_counts=True)
    giant = int(roots[np.argmax(sizes)])
    members = np.flatnonzero(lab == giant)
    srcs = gg.pick_seeded(members, COUNT, SRC_SEED)
    deg = g.degrees()
    with open(out, "w") as f:
        f.write("# Sources of the Kronecker scale-27 workload: 16 vertices drawn by seed 2 from the giant\n")
        f.write("# component (Sec. 5.2 averages over random sources); the component is the oracle's\n")
        f.write("# union-find label with the most vertices.  Written by make_kron27_sources.py.\n")
        f.write(f"scale {SCALE}\nedge_factor {EF}\ngen_seed {GEN_SEED}\nsrc_seed {SRC_SEED}\n")
        f.write(f"n {g.n}\nm {g.m}\ncomponents {roots.size}\ngiant_label {giant}\n")
        f.write(f"giant_vertices {members.size}\n")
        f.write(f"giant_directed_edges {int(deg[members].sum())}\n")
        f.write("sources " + " ".join(str(int(s)) for s in srcs) + "\n")
    print(f"wrote {out}: generation {t1 - t0:.0f} s, union-find {t2 - t1:.0f} s, "
          f"giant {members.size} of {g.n} vertices")


if __name__ == "__main__":
    main(*sys.argv[1:2])
