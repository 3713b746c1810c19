"""Pins of the learned-proposal oracle (network, training step, features)
against closed forms and finite differences."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def mlp():
    import oracle.mlp as m
    return m


def test_bf16_rounding_known_values(mlp):
    one = 1.0
    assert mlp.bf16(one) == 1.0
    assert mlp.bf16(1 + 2 ** -8) == 1.0                      # tie, even neighbour below
    assert mlp.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6          # tie, even neighbour above
    assert mlp.bf16(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7   # above the tie
    assert mlp.bf16(-3.0) == -3.0 and mlp.bf16(0.0) == 0.0


def test_closed_form_uniform_network(mlp):
    """All weights and biases zero except b4[32] = c: the PDF is uniform,
    T^ = sigmoid(c), the loss is mean(w (sum q log q + log 32) + (T^ - T)^2) and
    dL/db4[b] = mean(w (1/32 - q_b))."""
    p = np.zeros(synth.PROPOSAL_PARAMS)
    c = 0.7
    p[-40 + 32] = c
    f, t = synth.proposal_batch(4, 50)
    out = mlp.forward(p, f)
    np.testing.assert_allclose(out["pdf"], 1 / 32, atol=1e-15)
    np.testing.assert_allclose(out["that"], 1 / (1 + np.exp(-c)), atol=1e-15)
    loss, g = mlp.loss_and_grad(p, f, t)
    t = t.astype(np.float64)
    S = t[:, :32].sum(axis=1)
    q = np.where(S[:, None] > 0, t[:, :32] / np.where(S > 0, S, 1)[:, None], 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        qlogq = np.where(q > 0, q * np.log(np.where(q > 0, q, 1)), 0).sum(axis=1)
    sig = 1 / (1 + np.exp(-c))
    expect = np.mean(S * (qlogq + np.log(32) * (S > 0)) + (sig - t[:, 32]) ** 2)
    assert loss == pytest.approx(expect, rel=1e-12)
    gb4 = g[-40:]
    np.testing.assert_allclose(gb4[:32], np.mean(S[:, None] * (1 / 32 - q) * (S[:, None] > 0), axis=0), atol=1e-15)
    assert gb4[32] == pytest.approx(np.mean(2 * (sig - t[:, 32]) * sig * (1 - sig)), rel=1e-12)
    assert np.all(g[:-40] == 0)


def test_gradient_matches_finite_differences(mlp):
    p = synth.proposal_init_params(11).astype(np.float64)
    p += 0.01 * np.random.default_rng(0).normal(size=p.size) * (p != 0)   # non-zero biases
    f, t = synth.proposal_batch(5, 40)
    _, g = mlp.loss_and_grad(p, f, t, round_bf16=False)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(np.flatnonzero(g), 60, replace=False), np.argsort(-np.abs(g))[:20]])
    h = 1e-6
    for i in idx:
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (mlp.loss_and_grad(pp, f, t, False)[0] - mlp.loss_and_grad(pm, f, t, False)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_adam_first_step_is_signed_learning_rate(mlp):
    """With zero moments, Adam's first step is -lr g/(|g| + eps)."""
    g = np.array([1e-3, -2.0, 0.0, 5e-9])
    p, m, v = mlp.adam(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_features_of_an_axis_ray(orc):
    """Ray along -x through (y, z) = (3, 5) of a 64 x 8 x 12 box: entry point
    (1, 3/7, 5/11), direction (-1, 0, 0); encodings sin/cos(2^j pi x); the
    occupancy bits are those of the bricks the 32 bin centres fall in."""
    vol = np.zeros((12, 8, 64), dtype=np.uint16)
    vol[:, :, 20:30] = 3000                                  # tissue only in x-bricks 1
    tf = synth.tf_table(256)
    cam = dict(eye=(63.0 + 40.0, 3.0, 5.0), target=(0.0, 3.0, 5.0), up=(0.0, 0.0, 1.0), fovy_deg=30.0,
               width=1, height=1)
    sc = orc.Scene(vol, (1, 1, 1), tf, cam)
    mn, mx = orc.brick_minmax(vol)
    occ = orc.occupancy((64, 8, 12), tf, mn, mx)
    assert occ.ravel().tolist() == [0, 1, 0, 0]              # footprint 16..32 holds 20..29
    f = orc.proposal_features(sc, occ)[0]
    x = np.array([1.0, np.float32(3) / np.float32(7), np.float32(5) / np.float32(11), -1.0, 0.0, 0.0])
    np.testing.assert_allclose(f[:6], x, atol=1e-7)
    for c in range(6):
        for j in range(6):
            assert f[6 + 12 * c + 2 * j] == pytest.approx(np.sin(np.pi * 2 ** j * x[c]), abs=1e-6)
            assert f[7 + 12 * c + 2 * j] == pytest.approx(np.cos(np.pi * 2 ** j * x[c]), abs=1e-6)
    # bin b centre: x = 63 - (b + 0.5) * 63 / 32; cell-brick 1 holds cell bases 16..31
    centres = 63 - (np.arange(32) + 0.5) * 63 / 32
    expect = ((np.floor(centres) >= 16) & (np.floor(centres) < 32)).astype(float)
    np.testing.assert_array_equal(f[78:110], expect)
    assert f[110] == 0 and f[111] == 0


def test_missing_ray_has_zero_features(orc):
    vol = np.zeros((8, 8, 8), dtype=np.uint16)
    cam = dict(eye=(100.0, 100.0, 100.0), target=(200.0, 200.0, 200.0), up=(0.0, 0.0, 1.0),
               fovy_deg=30.0, width=4, height=4)
    sc = orc.Scene(vol, (1, 1, 1), synth.tf_table(256), cam)
    occ = np.ones((1, 1, 1), dtype=np.uint8)
    assert np.all(orc.proposal_features(sc, occ) == 0)
