"""Checkpoint / resume of a solve (gfcc_solve_checkpoint): every frequency's G block lands in the file
as it is solved; a rerun restores the finished frequencies and solves only the others (a job killed
while writing leaves a record cut short, which is dropped), and G equals the uninterrupted solve."""
import os

import numpy as np
import pytest

from paper_2010_04768_gb300 import gfcc
from paper_2010_04768_gb300.synthetic import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2010_04768_gb300 import build
    build.build()
    gfcc.load()


def test_resume_restores_finished_frequencies(tmp_path):
    o, v, L = 6, 24, 30
    pr = make_problem(o, v, L, seed=12)
    om = np.linspace(-1.0, -0.3, 5)
    orbs = np.array([o - 2, o - 1, o], dtype=np.int32)
    g = gfcc.GFCC(pr, sectors="IP+EA")
    G0, code0 = g.solve(om, 0.01, orbs, 1e-12)
    path = tmp_path / "g.ckpt"
    G1, code1, n1 = g.solve_checkpoint(om, 0.01, orbs, 1e-12, path)
    assert code0 == gfcc.OK and code1 == gfcc.OK and n1 == 0
    assert np.abs(G1 - G0).max() <= 1e-10 * np.abs(G0).max()
    # a job killed while writing the third record: two complete records and a piece of the third
    head = 8 + 5 * 4 + 2 * 8 + om.size * 8 + orbs.size * 4
    rec = 8 + 16 * orbs.size * orbs.size
    with open(path, "r+b") as f:
        f.truncate(head + 2 * rec + rec // 3)
    G2, code2, n2 = g.solve_checkpoint(om, 0.01, orbs, 1e-12, path)
    assert code2 == gfcc.OK and n2 == 2
    assert np.array_equal(G2[:2], G1[:2])                      # restored from the file as written
    assert np.abs(G2 - G0).max() <= 1e-10 * np.abs(G0).max()
    assert os.path.getsize(path) == head + om.size * rec     # the piece was dropped, all records now
    # everything restored: nothing solved
    G3, code3, n3 = g.solve_checkpoint(om, 0.01, orbs, 1e-12, path)
    assert n3 == om.size and np.array_equal(G3, G2)
    # a different request against the same file is refused and leaves it untouched
    size = os.path.getsize(path)
    with pytest.raises(gfcc.GFCCError):
        g.solve_checkpoint(om, 0.02, orbs, 1e-12, path)
    assert os.path.getsize(path) == size
    g.close()
