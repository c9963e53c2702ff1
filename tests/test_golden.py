"""The stored Green's function of the tiny workload (tests/golden/tiny_green_definition.txt, written
by tests/golden/make_tiny_green.py from the formula-free definition of oracle/fock_space.py) against
the scalable CPU oracle (CPU) and against the GPU path through the C ABI (FP64 and mixed precision)."""
import os

import numpy as np
import pytest

from paper_2010_04768_gb300.synthetic import workload

HERE = os.path.dirname(os.path.abspath(__file__))


def load_golden():
    omegas, entries = {}, []
    with open(os.path.join(HERE, "golden", "tiny_green_definition.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "omega":
                omegas[int(parts[1])] = float(parts[2])
            else:
                entries.append((int(parts[0]), int(parts[1]), int(parts[2]), float(parts[3]) + 1j * float(parts[4])))
    return np.array([omegas[k] for k in sorted(omegas)]), entries


def compare(G, entries):
    ref = np.array([g for *_, g in entries])
    got = np.array([G[w, p, q] for w, p, q, _ in entries])
    return np.abs(got - ref).max() / np.abs(ref).max()


def test_golden_file_matches_the_workload_and_the_scalable_oracle():
    from oracle.gfcc_ref import GFCCOracle
    wl = workload("tiny")
    omegas, entries = load_golden()
    assert np.array_equal(omegas, wl.omegas)
    assert len(entries) == omegas.size * (16 + 2 * 15)
    pr = wl.problem()
    G = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=wl.o).green_dense(wl.omegas, wl.eta, list(range(16)))
    assert compare(G, entries) <= 1e-11


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-12, 1e-10), ("mixed", 1e-10, 1e-6)])
def test_gpu_path_reproduces_the_golden_file(precision, tol, bar):
    from paper_2010_04768_gb300 import build, gfcc
    build.build()
    wl = workload("tiny")
    omegas, entries = load_golden()
    g = gfcc.GFCC(wl.problem(), precision=precision)
    G, code = g.solve(omegas, wl.eta, np.arange(16, dtype=np.int32), tol)
    g.close()
    assert code == gfcc.OK
    assert compare(G, entries) <= bar
