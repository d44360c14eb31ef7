"""Pins of the oracle pieces of the learned con2prim seeder (not part of the paper).

- The MLP backward (FP64, no rounding) against central finite differences of the loss.
- Closed forms: zero hidden weights give y = b4 and dL/db4 = 2 (b4 - mean t) / 3.
- One Adam step against the textbook update written out here.
- Seeded con2prim finds the same root as the plain bracket (the root is unique),
  uses the seed bracket when the seed is close, and falls back otherwise.
"""
import numpy as np

import oracle
import synth

NPAR = oracle.MLP_NPARAMS


def _params(rng, scale=0.3):
    return (scale * rng.normal(size=NPAR)).astype(np.float32)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = _params(rng)
    x = rng.normal(size=(16, 8)).astype(np.float32)
    t = rng.normal(size=(16, 3)).astype(np.float32)
    loss, g = oracle.mlp_grad(p, x, t, bf16=False)
    # Parameters are float32: perturb in float64 copies through a float64 path
    # by finite differences on the loss evaluated with the forward.
    def L(pp):
        y = oracle.mlp_forward(pp, x, bf16=False)
        return np.mean((y - t) ** 2)
    idx = rng.choice(NPAR, 40, replace=False)
    for q in idx:
        h = 2e-6 * max(1.0, abs(float(p[q])))  # small: no ReLU kink crossed
        pp, pm = p.copy(), p.copy()
        pp[q] += np.float32(h)
        pm[q] -= np.float32(h)
        hq = float(pp[q]) - float(pm[q])
        fd = (L(pp) - L(pm)) / hq
        assert abs(fd - g[q]) <= 1e-4 * max(1e-3, abs(g[q])) + 1e-7, (q, fd, g[q])
    assert abs(loss - L(p)) < 1e-12


def test_mlp_closed_forms():
    p = np.zeros(NPAR, dtype=np.float32)
    b4 = np.array([0.5, -1.0, 2.0], dtype=np.float32)
    p[-3:] = b4
    rng = np.random.default_rng(1)
    x = rng.normal(size=(10, 8)).astype(np.float32)
    t = rng.normal(size=(10, 3)).astype(np.float32)
    y = oracle.mlp_forward(p, x)
    assert np.allclose(y, b4[None, :])
    loss, g = oracle.mlp_grad(p, x, t)
    assert np.allclose(g[-3:], 2.0 * (b4.astype(float) - t.astype(float).mean(axis=0)) / 3.0, rtol=1e-12, atol=1e-12)
    assert np.all(g[:-3] == 0.0)  # ReLU of zero pre-activations blocks every other gradient


def test_adam_step():
    rng = np.random.default_rng(2)
    w, m, v, g = (rng.normal(size=50) for _ in range(4))
    v = np.abs(v)
    lr, b1, b2, eps, t = 1e-3, 0.9, 0.999, 1e-8, 3
    w2, m2, v2 = oracle.adam(w.copy(), m.copy(), v.copy(), g, lr, b1, b2, eps, t)
    mm = b1 * m + (1 - b1) * g
    vv = b2 * v + (1 - b2) * g * g
    ww = w - lr * (mm / (1 - b1 ** t)) / (np.sqrt(vv / (1 - b2 ** t)) + eps)
    assert np.allclose(w2, ww, rtol=1e-15, atol=1e-15) and np.allclose(m2, mm) and np.allclose(v2, vv)


def test_adam_bias_correction_on_a_constant_gradient():
    """Kingma & Ba's bias correction makes the moment estimates exact for a
    constant gradient started from zero moments: m_hat = g, v_hat = g^2 at
    every step t, so each step moves w by lr g / (|g| + eps) (about lr sign g,
    the step-size bound of the method)."""
    rng = np.random.default_rng(5)
    g = rng.normal(size=40) * 10 ** rng.uniform(-3, 1, 40)
    w0 = rng.normal(size=40)
    w, m, v = w0.copy(), np.zeros(40), np.zeros(40)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    step = lr * g / (np.abs(g) + eps)
    for t in range(1, 6):
        w, m, v = oracle.adam(w, m, v, g, lr, b1, b2, eps, t)
        assert np.allclose(w, w0 - t * step, rtol=0, atol=1e-13 * t)
        assert np.allclose(m / (1 - b1 ** t), g, rtol=1e-13)
        assert np.allclose(v / (1 - b2 ** t), g * g, rtol=1e-12)


def _cons(O, n, seed):
    s = synth.c2p_states(n, seed=seed)
    cons = np.zeros((n, 10))
    for q in range(n):
        pr = np.zeros(oracle.NP)
        pr[0], pr[7] = s["rho"][q], s["ye"][q]
        e = O.eos_from_T(s["rho"][q], s["T"][q], s["ye"][q])
        pr[1], pr[2] = e[1], e[0]
        pr[3:6] = s["v"][q]
        cons[q, :9] = oracle.prim2con_point(pr, s["B"][q], [1.0, 0, 0, 1.0, 0, 1.0])
    return cons


def test_seeded_con2prim_same_root_and_fallback():
    table = synth.make_table(nr=64, nt=48, ny=16)
    O = oracle.Oracle(synth.table_params(table), table)
    cons = _cons(O, 400, seed=5)
    p0, s0, it0, roots, _ = O.c2p_flat_ext(cons)
    ok = s0 >= 0
    # Close seeds: the seed brackets are used and the primitives agree to rounding.
    seeds = roots * (1.0 + 2e-4)
    p1, s1, it1, r1, sd = O.c2p_flat_ext(cons, seeds, delta=1e-3)
    assert np.array_equal(s0, s1)
    assert np.mean((sd[ok] & 2) > 0) > 0.9
    assert np.all(np.abs(p1[ok, 0] - p0[ok, 0]) <= 1e-13 * p0[ok, 0])
    assert np.all(np.abs(r1[ok, 1] - roots[ok, 1]) <= 1e-13 * roots[ok, 1])
    assert it1[ok].mean() < it0[ok].mean()
    # Unusable seeds (non-finite, negative, far off): the plain brackets, same result.
    bad = np.where(np.arange(400)[:, None] % 3 == 0, np.nan, np.where(np.arange(400)[:, None] % 3 == 1, -1.0, 1e3))
    bad = np.broadcast_to(bad, (400, 3)).copy()
    p2, s2, it2, r2, sd2 = O.c2p_flat_ext(cons, bad, delta=1e-3)
    assert np.all(sd2 == 0)
    assert np.array_equal(s2, s0) and np.array_equal(p2, p0)


def test_seeder_features_and_targets_closed_forms():
    # D = 1e-3, Ye = 0.1, q = 0.2, S = (1e-4, 0, 0) -> r = 0.1, B = (1e-3, 0, 0) -> b2 = 1e-3, S parallel to B.
    c = np.zeros((3, 10))
    c[:, 0], c[:, 1], c[:, 2] = 1e-3, 1e-4, 2e-4
    c[0, 3], c[0, 6] = 1e-4, 1e-3
    c[1, 3], c[1, 7] = 1e-4, 1e-3          # S perpendicular to B
    c[2, 3] = -1e-4                        # no field
    f = oracle.seeder_features(c)
    want = [-3.0, 0.1, np.log(1.2), np.log(1.1 * 1.3), 0.1 / 1.2, -3.0, 1.0, 1e-3 / 1.2]
    assert np.allclose(f[0], want, rtol=1e-14, atol=1e-15)
    assert abs(f[1, 6]) < 1e-15 and f[2, 5] == -30.0 and f[2, 6] == 0.0 and f[2, 7] == 0.0
    t = oracle.seeder_targets(c[:1], np.array([[0.5, 0.25, 3.0]]))
    assert np.allclose(t[0], [np.log(0.5 * np.sqrt(1.01)), np.log(0.25 * 1.2), np.log(3.0)], rtol=0, atol=1e-15)


def test_seeder_targets_vanish_for_the_unmagnetised_closed_forms():
    # B = 0 and h0 = 1: mu_+ = 1 / sqrt(1 + r^2) exactly, and mu (1 + q) = 1 - p / (rho h W^2).
    P = synth.ideal_params()
    assert P["h0"] == 1.0
    O = oracle.Oracle(P)
    rows, pr_list = [], []
    for rho, eps, v in [(1e-3, 0.1, 0.3), (1e-5, 2.0, 0.9), (0.1, 1e-4, 0.0), (1e-7, 5e-3, 0.99)]:
        pr = np.zeros(oracle.NP)
        pr[0], pr[1], pr[2], pr[3], pr[7] = rho, eps, rho * eps, v, 0.1
        c = np.zeros(10)
        c[:9] = oracle.prim2con_point(pr, [0, 0, 0], [1.0, 0, 0, 1.0, 0, 1.0])
        rows.append(c)
        pr_list.append(pr)
    cons = np.array(rows)
    p, st, _, roots, _ = O.c2p_flat_ext(cons)
    assert np.all(st == 0)
    t = oracle.seeder_targets(cons, roots)
    assert np.all(np.abs(t[:, 0]) <= 2e-15)
    for k, pr in enumerate(pr_list):
        rho, eps, prs, v = pr[0], pr[1], pr[2], pr[3]
        W = 1.0 / np.sqrt(1.0 - v * v)
        h = 1.0 + eps + prs / rho
        assert abs(t[k, 1] - np.log(1.0 - prs / (rho * h * W * W))) <= 1e-12
        assert abs(t[k, 2] - np.log(W)) <= 1e-12
