"""GPU parity of the spectral correction and its learned model against the
FP64 oracle: exact targets, the model's forward pass, training steps, the
corrected preconditioner (exact and learned delta) and restoration with a
prebuilt preconditioner.  Model parameters are seeded numpy draws shared by
both sides.  Bounds: float64 setup 1e-12; float32 forward passes (sums of at
most 256 products) 2e-5 relative to the output scale; restoration tol(alpha)
as in test_gpu_parity."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1211_0393_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ar():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0393_gb300 import ar as mod

    mod.lib()
    return mod


def flat(P):
    return np.concatenate([P[k].reshape(-1) for k in O.PARAM_ORDER]).astype(np.float32)


def unflat(v):
    shapes = {"W1": (225, 256), "b1": (256,), "W2": (256, 256), "b2": (256,), "W3": (256, 1089),
              "b3": (1089,)}
    P, o = {}, 0
    for k in O.PARAM_ORDER:
        n = int(np.prod(shapes[k]))
        P[k] = v[o:o + n].astype(np.float64).reshape(shapes[k])
        o += n
    return P


def psfs(seed, count):
    rng = np.random.default_rng(seed)
    return np.stack([W.psf_random(7, 7, rng) for _ in range(count)])


def model_params(seed):
    P = O.mlp_init(np.random.default_rng(seed))
    rng = np.random.default_rng(seed + 1)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(0, 0.05, P[k].shape)
    # store in float32 and read back so both sides hold the same values
    return unflat(flat(P))


def test_targets_match_oracle(ar):
    H = psfs(1, 6)
    got = ar.corr_targets(H)
    for i in range(len(H)):
        want = O.corr_target(H[i])
        assert np.max(np.abs(got[i] - want)) <= 1e-13 * max(1.0, np.max(want))


def test_forward_matches_oracle(ar):
    P = model_params(3)
    M = ar.Corr(flat(P))
    for h in psfs(4, 4):
        got = M.predict(h)
        Y, _ = O.mlp_forward(P, O.corr_input(h)[None, :])
        want = Y[0].reshape(33, 33)
        assert np.max(np.abs(got - want)) <= 2e-5 * np.max(np.abs(want))
    M.close()


def test_training_steps_match_oracle(ar):
    """Two epochs over one batch: the first loss is the initial model's, the
    second follows one Adam step, on both sides."""
    P = model_params(5)
    H = psfs(6, 8)
    M = ar.Corr(flat(P))
    loss = M.train(H, epochs=2, batch=8, lr=1e-3)
    X = np.stack([O.corr_input(h) for h in H])
    T = np.stack([O.corr_target(h).reshape(-1) for h in H])
    Y, cache = O.mlp_forward(P, X)
    l0, dY = O.mse_loss(Y, T)
    st = {}
    O.adam_step(P, O.mlp_backward(P, cache, dY), st, lr=1e-3)
    l1, _ = O.mse_loss(O.mlp_forward(P, X)[0], T)
    assert loss[0] == pytest.approx(l0, rel=1e-5)
    assert loss[1] == pytest.approx(l1, rel=1e-3)
    assert loss[1] < loss[0]
    M.close()


def test_adam_steps_match_oracle_elementwise(ar):
    """Every parameter after six Adam steps (three epochs of two batches, taken in
    order) against the oracle's forward pass, backward pass and Adam update.

    Adam normalises each update by the running gradient scale, so an entry whose
    gradient is at the float32 rounding level of its tensor (or whose ReLU mask
    flips on a pre-activation at rounding level) can move by up to lr per step in
    either direction on either side.  Entries whose oracle gradient stays above
    1e-3 of the tensor's largest at every step are determined by the arithmetic
    and must agree to 2e-5 (float32 gradients carry relative errors of about 1e-3
    there, on updates of size lr = 1e-3; a float32 emulation of the training
    agrees to 4e-8 on them and to 1.1e-6 on all entries).  All but 0.1% of every
    tensor must agree to 2e-5 as well (exactly-zero gradients of inactive units
    are zero on both sides), and no entry may differ by more than the Adam step
    bound, 2 lr per step.  A wrong gradient of any layer, a wrong bias
    correction or a wrong moment update moves the determined entries by about
    lr and fails."""
    P = model_params(5)
    H = psfs(6, 16)
    lr, epochs, batch = 1e-3, 3, 8
    M = ar.Corr(flat(P))
    loss = M.train(H, epochs=epochs, batch=batch, lr=lr)
    got = unflat(M.params())
    M.close()
    X = np.stack([O.corr_input(h) for h in H])
    T = np.stack([O.corr_target(h).reshape(-1) for h in H])
    Po = {k: v.copy() for k, v in P.items()}
    st = {}
    minrel = {k: np.full(v.shape, np.inf) for k, v in P.items()}
    steps = 0
    for _ in range(epochs):
        for b0 in range(0, len(H), batch):
            Y, cache = O.mlp_forward(Po, X[b0:b0 + batch])
            _, dY = O.mse_loss(Y, T[b0:b0 + batch])
            G = O.mlp_backward(Po, cache, dY)
            for k in O.PARAM_ORDER:
                minrel[k] = np.minimum(minrel[k], np.abs(G[k]) / np.max(np.abs(G[k])))
            O.adam_step(Po, G, st, lr=lr)
            steps += 1
    assert steps == 6 and len(loss) == epochs
    for k in O.PARAM_ORDER:
        d = np.abs(got[k] - Po[k])
        det = minrel[k] >= 1e-3
        assert det.mean() >= 0.1, (k, det.mean())
        assert np.max(d[det]) <= 2e-5, (k, np.max(d[det]))
        assert np.mean(d > 2e-5) <= 1e-3, (k, np.mean(d > 2e-5))
        assert np.max(d) <= 2 * lr * steps, (k, np.max(d))
        # the parameters really moved: the comparison is not of two initial states
        assert np.median(np.abs(Po[k] - P[k])[det]) > 0.5 * lr


@pytest.mark.parametrize("n1,n2", [(64, 64), (33, 33), (130, 97)])
def test_exact_corrected_setup_matches_oracle(ar, n1, n2):
    h = W.psf_config2()
    P = ar.ar_symprec_setup_corrected(h, n1, n2, 0.1)
    lam, d = ar.ar_symprec_eigenvalues(P)
    prec = O.symprec_setup_corrected(h, n1, n2, 0.1)
    assert np.max(np.abs(lam - prec["lam"])) <= 1e-13
    assert np.max(np.abs(d - prec["d"]) / prec["d"]) <= 1e-12
    P.close()


def test_learned_corrected_setup_matches_oracle(ar):
    Pm = model_params(7)
    M = ar.Corr(flat(Pm))
    h = W.psf_config2()
    P = ar.ar_symprec_setup_corrected(h, 96, 80, 0.1, model=M)
    _, d = ar.ar_symprec_eigenvalues(P)
    want = O.symprec_setup_corrected(h, 96, 80, 0.1, table=O.mlp_predict_table(Pm, h))["d"]
    assert np.max(np.abs(d - want) / want) <= 1e-5
    P.close()
    M.close()


def _workload(n, h, cidx, nu):
    q1, q2 = O.psf_support(h)
    ext, f, e = W.make_inputs(n, n, h, "ellipses", cidx)
    g = W.add_noise(W.crop(O.ar_blur(ext, h), q1, q2), e, nu)
    return g.astype(np.float32), f.astype(np.float32)


def test_restore_with_corrected_preconditioner_matches_oracle(ar):
    h = W.psf_config2()
    g, f = _workload(128, h, 1, 0.005)
    P = ar.ar_symprec_setup_corrected(h, 128, 128, 0.1)
    x, tr, best = ar.ar_restore_prec(P, torch.from_numpy(g).cuda(), h, 1.0, 8,
                                     f_true=torch.from_numpy(f).cuda())
    xo, to, bo = O.restore_corrected(g.astype(np.float64), h, 0.1, 1.0, 8,
                                     f_true=f.astype(np.float64))
    tol = max(1e-5, 3 * 2.0 ** -24 / 0.1)
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= tol
    assert np.all(np.abs(tr - to) <= tol * (1 + to))
    P.close()


def test_restore_prec_with_symmetrized_preconditioner_equals_restore(ar):
    h = W.psf_config2()
    g, f = _workload(128, h, 1, 0.005)
    gd, fd = torch.from_numpy(g).cuda(), torch.from_numpy(f).cuda()
    P = ar.ar_symprec_setup(h, 128, 128, 0.3)
    x1, t1, b1 = ar.ar_restore_prec(P, gd, h, 1.0, 6, f_true=fd)
    x2, t2, b2 = ar.ar_restore(gd, h, 0.3, 1.0, 6, True, f_true=fd)
    # the iterates are bit-identical; the RRE sums are float64 atomics (order varies)
    assert torch.equal(x1, x2) and b1 == b2
    np.testing.assert_allclose(t1, t2, rtol=1e-12, atol=0)
    P.close()


def test_restoration_targets_match_oracle(ar):
    """Tables read off the symmetrized D-Landweber's own iterates (GPU) against the
    oracle's on the same seeded scene, noise field and PSFs.  Bound: a frequency's
    shrunk departure (mu^ - lambda^2) w / (w + rho) moves by at most about
    e sqrt(K) / (tau d sqrt(rho)) when its spectral values W_k carry an absolute
    error e; float32 transforms give e ~ 2^-24 x the largest |W| (sums with
    cancellation); rho = 5 w_mean, and a 64^2 scene's largest weight is about
    1e3 w_mean, so rho >= 5e-3 max|W|^2 K; with K = 6 and tau d >= 1/(1 + 0.3)
    that is about 5e-6 per frequency, and a node is a weighted mean of them;
    checked at 1e-4."""
    n = 64
    rng = np.random.default_rng(21)
    f = rng.uniform(0, 1, (n, n)).astype(np.float32)
    e = rng.standard_normal((n, n)).astype(np.float32)
    H = psfs(22, 3)
    got = ar.corr_restoration_targets(torch.from_numpy(f).cuda(), torch.from_numpy(e).cuda(), H,
                                      0.005, 0.3, 1.0, 6)
    assert got.shape == (3, 33, 33)
    for i in range(3):
        want = O.restoration_target(H[i], f.astype(np.float64), e.astype(np.float64), 0.005, 0.3,
                                    1.0, 6)
        assert np.max(np.abs(got[i] - want)) <= 1e-4, (i, np.max(np.abs(got[i] - want)))
        assert np.max(np.abs(want)) > 1e-2            # a nonzero target is compared


def test_restoration_targets_vanish_for_a_symmetric_psf(ar):
    """Theorem 2 with A' = A: a strongly symmetric PSF leaves no departure to fit."""
    n = 48
    rng = np.random.default_rng(23)
    a = np.arange(-7, 8)
    h = np.exp(-0.5 * (a[:, None] ** 2 / 3.0 + a[None, :] ** 2 / 5.0))
    h = (h / h.sum())[None]
    f = torch.from_numpy(rng.uniform(0, 1, (n, n)).astype(np.float32)).cuda()
    e = torch.from_numpy(rng.standard_normal((n, n)).astype(np.float32)).cuda()
    got = ar.corr_restoration_targets(f, e, h, 0.01, 0.3, 1.0, 6)
    assert np.max(np.abs(got)) <= 1e-4


def test_training_on_given_tables_matches_oracle(ar):
    """ar_corr_train_tables: the first loss is the initial model's against the given
    tables, and the parameters after one Adam step follow the oracle's (the
    determined entries as in test_adam_steps_match_oracle_elementwise)."""
    P = model_params(9)
    H = psfs(10, 8)
    T = np.random.default_rng(11).normal(0.0, 0.1, (8, 33, 33))
    M = ar.Corr(flat(P))
    loss = M.train(H, epochs=1, batch=8, lr=1e-3, tables=T)
    got = unflat(M.params())
    M.close()
    X = np.stack([O.corr_input(h) for h in H])
    Tt = T.reshape(8, -1).astype(np.float32).astype(np.float64)
    Y, cache = O.mlp_forward(P, X)
    l0, dY = O.mse_loss(Y, Tt)
    G = O.mlp_backward(P, cache, dY)
    Po = {k: v.copy() for k, v in P.items()}
    O.adam_step(Po, G, {}, lr=1e-3)
    assert loss[0] == pytest.approx(l0, rel=1e-5)
    for k in O.PARAM_ORDER:
        det = np.abs(G[k]) >= 1e-3 * np.max(np.abs(G[k]))
        assert np.max(np.abs(got[k] - Po[k])[det]) <= 2e-5, k
