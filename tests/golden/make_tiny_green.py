"""Writes tiny_green_definition.txt: G_pq(omega) of eq. gfxn3 (G = G^IP + G^EA, eqs. gfxn1 / gfxn2)
for the tiny synthetic workload, computed by the formula-free definition in oracle/fock_space.py
(Fock-space operators, Hbar = e^-T H e^T applied to determinants, the shifted systems of eq. xplin
solved densely).  Only oracle/ and the seeded input generator are used.

    python tests/golden/make_tiny_green.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2010_04768_gb300.synthetic import workload  # noqa: E402
from oracle.fock_space import BruteForceGFCC  # noqa: E402

ROWS = (3, 4)   # full rows p = HOMO and p = LUMO; every diagonal element besides


def main():
    wl = workload("tiny")
    pr = wl.problem()
    bf = BruteForceGFCC(pr.fock, pr.chol, pr.t1, pr.t2, pr.t1, pr.t2, wl.o)   # Lambda = T^dagger
    orbs = list(range(wl.o + wl.v))
    G = bf.green_ip(wl.omegas, wl.eta, orbs) + bf.green_ea(wl.omegas, wl.eta, orbs)
    lines = [
        "# G_pq(omega) = G^IP + G^EA (eqs. gfxn1-gfxn3) of the tiny synthetic workload: o=4 v=12 L=48,",
        "# seed 0 (paper_2010_04768_gb300.synthetic.workload('tiny')), eta = %.17g, Lambda = T^dagger," % wl.eta,
        "# from the formula-free definition (oracle/fock_space.py: <mu|[Hbar, R_nu]|Phi>, eq. xplin solved",
        "# densely); written by tests/golden/make_tiny_green.py.  Columns: omega index, p, q, Re G, Im G.",
        "# Entries: every diagonal element and the full rows p = %s." % ", ".join(map(str, ROWS)),
    ]
    lines += ["omega %d %.17g" % (w, om) for w, om in enumerate(wl.omegas)]
    for w in range(len(wl.omegas)):
        for p in orbs:
            for q in orbs:
                if p == q or p in ROWS:
                    lines.append("%d %d %d %.17g %.17g" % (w, p, q, G[w, p, q].real, G[w, p, q].imag))
    with open(os.path.join(HERE, "tiny_green_definition.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
