"""Initial guesses and the learned-guess model on the GPU, against the CPU oracle (oracle/mlp_ref.py).

* model kernels: inference (FP64; FP16 weights), loss and gradient (FP64 vs the oracle's analytic
  gradient and vs FP64 finite differences of the oracle loss; FP32 vs finite differences), Adam steps;
* sample collection: Gram matrices and features of the kept solutions vs the oracle's dense solutions;
* guessed solves: G unchanged (to the solver tolerance), the predicted residual of each guess equal to
  the measured first residual, the guess of each system equal to the oracle's replay of the same
  schedule, fewer iterations than the zero guess, and a trained model that beats the zero guess on a
  held-out problem.
"""
import numpy as np
import pytest

from oracle import mlp_ref as M
from oracle.gfcc_ref import GFCCOracle
from paper_2010_04768_gb300 import gfcc
from paper_2010_04768_gb300.synthetic import make_problem, mlp_init_params, orbitals_nearest_gap

pytestmark = pytest.mark.gpu

O, V, L = 6, 24, 48
ETA = 0.01


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2010_04768_gb300 import build
    build.build()
    gfcc.load()


def problem(seed):
    pr = make_problem(O, V, L, seed=seed)
    eps = np.diag(pr.fock)
    return pr, orbitals_nearest_gap(eps[:O], eps[O:], 4)


def dense_solutions(orc, Mip, b, omegas):
    n = Mip.shape[0]
    return np.stack([np.linalg.solve((w - 1j * ETA) * np.eye(n) + Mip, b) for w in omegas])


def random_samples(rng, count):
    F = rng.normal(size=(count, 27))
    Gms = []
    for _ in range(count):
        U = rng.normal(size=(9, 20)) + 1j * rng.normal(size=(9, 20))
        Gms.append(U.conj() @ U.T)
    return F, np.array(Gms)


def model_params(hidden, seed, rng):
    flat = mlp_init_params(hidden, seed)
    nparam = flat.size
    flat[nparam - 54:nparam - 27] = 0.1 * rng.normal(size=27)
    flat[nparam - 27:] = 0.5 + rng.uniform(size=27)
    return flat


# ------------------------------------------------------------------------------------ model kernels

def test_forward_fp64_matches_oracle():
    rng = np.random.default_rng(0)
    flat = model_params(256, 1, rng)
    m = gfcc.MLP(flat, 256, gfcc.MLP_FP64)
    m.set_params(flat)
    F, _ = random_samples(rng, 37)
    y = m.forward(F)
    ref = M.MLPRef(flat, 256).forward(F)[-1]
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.array_equal(m.get_params(), flat)


def test_forward_fp16_weights_matches_rounded_oracle():
    rng = np.random.default_rng(1)
    flat = model_params(256, 2, rng)
    m = gfcc.MLP(flat, 256, gfcc.MLP_FP32)
    m.set_params(flat)
    F, _ = random_samples(rng, 19)
    y = m.forward(F)
    # the inference copy: weights rounded to FP16 (nearest even), vectors to FP32
    net = M.MLPRef(flat, 256)
    W1, b1, W2, b2, W3, b3, mu, sd = net.unpack()
    r = []
    for a, half in ((W1, 1), (b1, 0), (W2, 1), (b2, 0), (W3, 1), (b3, 0), (mu, 0), (sd, 0)):
        r.append(a.astype(np.float16 if half else np.float32).astype(np.float64).ravel())
    rnet = M.MLPRef(np.concatenate(r), 256)
    ref = rnet.forward(F)[-1]
    # A-priori bound of the FP32 evaluation (both sides use the same FP16 weights): the input
    # (x - mu) / sd is rounded once to FP32 (|dx| <= u |x|); each layer z = b + W h sums n terms in FP32
    # (fused or not, any order), so |fl(z) - z| <= |W| e_in + gamma_n (|b| + |W| (|h| + e_in)) with
    # gamma_n = n u / (1 - n u), u = 2^-24 (Higham, Accuracy and Stability of Numerical Algorithms, 3.1);
    # ReLU is 1-Lipschitz, so the bound e of a layer's output is the input bound of the next.
    u = 2.0 ** -24
    gam = lambda n: n * u / (1 - n * u)
    W1r, b1r, W2r, b2r, W3r, b3r, mur, sdr = rnet.unpack()
    xh = (F - mur) / sdr
    h1 = np.maximum(xh @ W1r.T + b1r, 0.0)
    h2 = np.maximum(h1 @ W2r.T + b2r, 0.0)
    e0 = u * np.abs(xh)
    e1 = e0 @ np.abs(W1r).T + gam(W1r.shape[1]) * (np.abs(b1r) + (np.abs(xh) + e0) @ np.abs(W1r).T)
    e2 = e1 @ np.abs(W2r).T + gam(W2r.shape[1]) * (np.abs(b2r) + (h1 + e1) @ np.abs(W2r).T)
    e3 = e2 @ np.abs(W3r).T + gam(W3r.shape[1]) * (np.abs(b3r) + (h2 + e2) @ np.abs(W3r).T)
    assert np.all(np.abs(y - ref) <= e3 + 1e-12 * np.abs(ref))
    ref64 = net.forward(F)[-1]
    assert np.max(np.abs(y - ref64)) <= 5e-3 * np.max(np.abs(ref64))


def test_loss_and_gradient_fp64_match_oracle_and_finite_differences():
    rng = np.random.default_rng(2)
    hidden = 64
    flat = model_params(hidden, 3, rng)
    m = gfcc.MLP(flat, hidden, gfcc.MLP_FP64)
    m.set_params(flat)
    F, Gms = random_samples(rng, 24)
    loss, g = m.loss_grad(F, Gms)
    net = M.MLPRef(flat, hidden)
    loss_ref, g_ref = net.loss_and_grad(F, Gms)
    assert loss == pytest.approx(loss_ref, rel=1e-12)
    assert np.max(np.abs(g - g_ref)) <= 1e-11 * np.max(np.abs(g_ref))
    h = 1e-6
    for i in rng.choice(flat.size - 54, size=25, replace=False):
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        fd = (M.MLPRef(fp, hidden).loss(F, Gms) - M.MLPRef(fm, hidden).loss(F, Gms)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-8 * np.max(np.abs(g_ref)) + 1e-8 * abs(fd)


def test_gradient_fp32_matches_finite_differences():
    rng = np.random.default_rng(3)
    hidden = 64
    flat = model_params(hidden, 4, rng)
    m = gfcc.MLP(flat, hidden, gfcc.MLP_FP32)
    # FP32 master copy: compare against the oracle at the FP32-rounded parameters
    flat32 = flat.astype(np.float32).astype(np.float64)
    m.set_params(flat32)
    F, Gms = random_samples(rng, 24)
    _, g = m.loss_grad(F, Gms)
    _, g_ref = M.MLPRef(flat32, hidden).loss_and_grad(F, Gms)
    assert np.max(np.abs(g - g_ref)) <= 1e-3 * np.max(np.abs(g_ref))
    h = 1e-6
    for i in rng.choice(flat.size - 54, size=10, replace=False):
        fp, fm = flat32.copy(), flat32.copy()
        fp[i] += h
        fm[i] -= h
        fd = (M.MLPRef(fp, hidden).loss(F, Gms) - M.MLPRef(fm, hidden).loss(F, Gms)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-3 * np.max(np.abs(g_ref))


def test_adam_steps_fp64_match_oracle():
    rng = np.random.default_rng(4)
    hidden = 32
    flat = model_params(hidden, 5, rng)
    m = gfcc.MLP(flat, hidden, gfcc.MLP_FP64)
    m.set_params(flat)
    net_flat = flat.copy()
    opt = M.AdamRef(flat.size - 54)
    for step in range(3):
        F, Gms = random_samples(rng, 16)
        loss = m.train_batch(F, Gms, lr=1e-3)
        loss_ref, g_ref = M.MLPRef(net_flat, hidden).loss_and_grad(F, Gms)
        assert loss == pytest.approx(loss_ref, rel=1e-12)
        net_flat = opt.step(net_flat, g_ref, 1e-3)
    p = m.get_params()
    assert np.max(np.abs(p - net_flat)) <= 1e-10 * np.max(np.abs(net_flat))


# --------------------------------------------------------------------------- guessed solves

@pytest.fixture(scope="module")
def held_out():
    pr, orbs = problem(1000)
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=O, sectors=("IP",))
    return pr, orbs, orc, orc.ip_matrix()


def solve(pr, orbs, omegas, guess, model=None, keep=False, tol=1e-10):
    g = gfcc.GFCC(pr, sectors="IP")
    g.set_option(gfcc.OPT_BATCH, len(orbs))       # one frequency per batch: guesses from earlier batches
    g.set_option(gfcc.OPT_GUESS, guess)
    g.set_option(gfcc.OPT_KEEP_SOLUTIONS, 1 if keep else 0)
    if model is not None:
        g.set_guess_model(model)
    G, code = g.solve(omegas, ETA, orbs, tol)
    assert code == gfcc.OK
    it, rr, st = g.stats()
    kind, pred, rel0 = g.guess_stats()
    return g, G, it, kind, pred, rel0


def test_minres_guess_parity_and_gain(held_out):
    pr, orbs, orc, Mip = held_out
    omegas = np.linspace(-1.0, 0.4, 24)
    _, G0, it0, kind0, _, rel00 = solve(pr, orbs, omegas, gfcc.GUESS_ZERO)
    assert np.all(kind0 == 0) and np.allclose(rel00, 1.0)
    _, G1, it1, kind, pred, rel0 = solve(pr, orbs, omegas, gfcc.GUESS_MINRES)
    ref = orc.green_dense(omegas, ETA, orbs, sectors=("IP",))
    assert np.abs(G1 - ref).max() <= 1e-9 * np.abs(ref).max()
    assert np.abs(G1 - G0).max() <= 1e-9 * np.abs(ref).max()
    # the two ends go first with no neighbours; later frequencies are guessed
    order = M.frequency_order(omegas)
    no = len(orbs)
    kind_w = kind.reshape(len(omegas), no)
    assert np.all(kind_w[order[0]] == 0)
    assert np.mean(kind == gfcc.GUESS_MINRES) >= 0.8
    # predicted residual of the guess == measured first residual (up to the FP32 storage of X_k)
    g_idx = kind == gfcc.GUESS_MINRES
    assert np.all(np.abs(np.sqrt(pred[g_idx]) - rel0[g_idx]) <= 1e-4 + 1e-2 * rel0[g_idx])
    assert np.all(rel0[g_idx] < 1.0)
    assert it1.sum() < 0.8 * it0.sum()
    # replay of the schedule with the oracle: same neighbours, Gram from dense FP64 solutions
    pred_w = pred.reshape(len(omegas), no)
    for a, p in enumerate(orbs):
        b = orc.ip_rhs(int(p))
        X = dense_solutions(orc, Mip, b, omegas)
        done = np.zeros(len(omegas), dtype=bool)
        for w in order:
            nb = M.neighbours(omegas, done, w)
            Gm = M.gram(b, X[nb], omegas[w] - omegas[nb]) if nb else np.zeros((1, 1))
            if nb:
                Gm9 = np.zeros((9, 9), dtype=complex)
                Gm9[: len(nb) + 1, : len(nb) + 1] = Gm
                c, loss, k = M.choose(Gm9, len(nb), 2)
            else:
                loss, k = 1.0, 0
            assert kind_w[w, a] == k
            if k and loss > 1e-6:
                assert pred_w[w, a] == pytest.approx(loss, rel=5e-2)
            done[w] = True


def test_collected_samples_match_oracle(held_out):
    pr, orbs, orc, Mip = held_out
    omegas = np.linspace(-1.0, 0.4, 20)
    g, *_ = solve(pr, orbs, omegas, gfcc.GUESS_ZERO, keep=True)
    m = gfcc.MLP(mlp_init_params(64, 1), 64)
    added = m.collect(g, samples_per_system=1, seed=7)
    assert added == m.num_samples() and added > 0
    F, Gm = m.samples()
    n_orb_total = O + V
    Xcache = {}
    rng = np.random.default_rng(0)
    for s in rng.choice(added, size=min(12, added), replace=False):
        f = F[s]
        w = int(np.argmin(np.abs(omegas - f[0])))
        assert f[1] == ETA
        p = int(round(f[2] * n_orb_total))
        assert p in orbs
        nb = [int(np.argmin(np.abs(omegas - (f[0] - d)))) for d in f[3:11]]
        assert len(set(nb)) == 8 and w not in nb
        if p not in Xcache:
            Xcache[p] = (orc.ip_rhs(p), dense_solutions(orc, Mip, orc.ip_rhs(p), omegas))
        b, X = Xcache[p]
        ref = M.gram(b, X[nb], omegas[w] - omegas[nb])
        assert np.abs(Gm[s] - ref).max() <= 1e-6 * np.abs(ref).max()
        ov = np.array([np.vdot(b, X[k]) for k in nb]) * ETA / np.vdot(b, b).real
        assert np.allclose(f[11:19], ov.real, rtol=1e-5, atol=1e-7 * np.abs(ov).max())
        assert np.allclose(f[19:27], ov.imag, rtol=1e-5, atol=1e-7 * np.abs(ov).max())


def test_learned_guess_beats_zero_guess_on_a_held_out_problem(held_out):
    # training data: the method's own converged solutions of two other problems of the same shape
    model = gfcc.MLP(mlp_init_params(256, 0), 256, gfcc.MLP_FP32)
    omegas = np.linspace(-1.0, 0.4, 48)
    for seed in (1, 2):
        pr, orbs = problem(seed)
        g, *_ = solve(pr, orbs, omegas, gfcc.GUESS_ZERO, keep=True)
        model.collect(g, samples_per_system=3, seed=seed)
        g.close()
    loss = model.train(steps=1500, minibatch=128, lr=1e-3, seed=3)
    ev = model.eval()
    assert ev["frac_better_than_zero"] > 0.6 and ev["loss_fallback"] < 0.5
    assert ev["loss_minres"] <= ev["loss_fallback"]
    pr, orbs, orc, Mip = held_out
    _, G0, it0, *_ = solve(pr, orbs, omegas, gfcc.GUESS_ZERO)
    _, G1, it1, kind, pred, rel0 = solve(pr, orbs, omegas, gfcc.GUESS_LEARNED, model=model)
    assert np.abs(G1 - G0).max() <= 1e-9 * np.abs(G0).max()
    learned = kind == gfcc.GUESS_LEARNED
    assert learned.mean() >= 0.4
    assert np.all(pred[learned] < 1.0) and np.all(rel0[learned] < 1.0)
    assert it1.sum() < it0.sum()
    print(f"learned guess: train loss {loss:.3e}, eval {ev}, iterations {it1.sum()} vs zero guess {it0.sum()}, "
          f"guessed {learned.mean():.2f}, median predicted residual^2 {np.median(pred[learned]):.2e}")
