"""Pins of the network oracle (oracle/unet.py): the convolution against a
brute-force sum of its definition, pooling and upsampling against their
definitions, BF16 rounding against torch's conversion, the gradient against
central finite differences, and the all-zero network's closed form."""
import numpy as np
import pytest
import torch

from oracle import unet as U


def he_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = []
    for ci, co in U.LAYERS:
        p.append(rng.standard_normal(27 * ci * co) * scale * np.sqrt(2.0 / (27 * ci)))
        p.append(0.01 * rng.standard_normal(co))
    p.append(rng.standard_normal(16) * 0.25)
    p.append([0.1])
    return np.concatenate(p).astype(np.float32)


def test_conv_matches_definition():
    rng = np.random.default_rng(0)
    S, ci, co = 4, 3, 2
    x = rng.standard_normal((ci, S, S, S))
    W = rng.standard_normal(co * 27 * ci)
    b = rng.standard_normal(co)
    got = U.conv3(torch.from_numpy(x), U.conv_weight(W, ci, co), torch.from_numpy(b)).numpy()
    Wr = W.reshape(co, 27, ci)
    want = np.zeros((co, S, S, S))
    for o in range(co):
        for z in range(S):
            for y in range(S):
                for xx in range(S):
                    s = b[o]
                    for t in range(27):
                        dz, dy, dx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
                        zz, yy, x2 = z + dz, y + dy, xx + dx
                        if 0 <= zz < S and 0 <= yy < S and 0 <= x2 < S:
                            s += np.dot(Wr[o, t], x[:, zz, yy, x2])
                    want[o, z, y, xx] = s
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_pool_and_up():
    rng = np.random.default_rng(1)
    a = torch.from_numpy(rng.standard_normal((2, 4, 4, 4)))
    p = U.pool(a)
    assert p[1, 1, 0, 1].item() == pytest.approx(a[1, 2:4, 0:2, 2:4].mean().item(), rel=1e-14)
    u = U.up(p)
    assert u[0, 3, 1, 2].item() == p[0, 1, 0, 1].item()
    c = torch.from_numpy(rng.standard_normal((2, 4, 4, 4)))
    # nearest upsampling is 8 x the adjoint of average pooling
    assert torch.sum(U.up(p) * c).item() == pytest.approx(8.0 * torch.sum(p * U.pool(c)).item(), rel=1e-12)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5e-3, 3.3e4, 1.0 - 2.0 ** -10], dtype=np.float32)
    want = torch.from_numpy(vals).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(U.bf16_round(vals), want)
    assert U.bf16_round(np.float32([1.0 + 2.0 ** -8]))[0] == 1.0               # tie to even
    assert U.bf16_round(np.float32([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_layout_covers_vector():
    sl = U.layer_slices()
    assert sl[0][1].start == 0 and sl[-1][1].stop == U.num_params() == 1466065
    assert all(a[1].stop == b[1].start for a, b in zip(sl, sl[1:]))


def test_zero_network_closed_form():
    p = np.zeros(U.num_params(), dtype=np.float32)
    p[-1] = 0.5
    rng = np.random.default_rng(2)
    smp = rng.standard_normal(3 * 16 ** 3)
    loss, g = U.loss_and_gradients(p, [smp], [0.0])
    t = smp[2 * 16 ** 3:]
    assert loss == pytest.approx(np.mean((0.5 - t) ** 2), rel=1e-12)
    assert g[-1] == pytest.approx(2.0 * np.mean(0.5 - t), rel=1e-12)
    assert np.all(g[:-1] == 0.0)


def test_gradient_finite_differences():
    p = he_params(3).astype(np.float64)
    rng = np.random.default_rng(4)
    S = 16
    smp = [np.concatenate([rng.random(S ** 3), rng.standard_normal(S ** 3), 0.1 * rng.standard_normal(S ** 3)])
           for _ in range(2)]
    flags = [0.0, 1.0]
    _, g = U.loss_and_gradients(p, smp, flags, round_weights=False)
    picks = []
    for name, sl in U.layer_slices():
        idx = np.arange(sl.start, sl.stop)
        picks.append(int(idx[np.argmax(np.abs(g[idx]))]))  # the largest entry of each block
    for i in picks:
        eps = 1e-6 * max(1.0, abs(p[i]))  # small enough that no ReLU changes sign
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        lp, _ = U.loss_and_gradients(pp, smp, flags, round_weights=False)
        lm, _ = U.loss_and_gradients(pm, smp, flags, round_weights=False)
        fd = (lp - lm) / (2 * eps)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), (i, fd, g[i])


def test_bf16_activation_storage_closed_form():
    # all weights zero: every convolution outputs relu(bias), so the output is
    # sum_c w_c relu(b13_c) + b_head with the last layer's activations stored
    # in BF16 (1 + 2^-10 and 3 + 2^-7 are not BF16 values; 1 and 3 are)
    p = np.zeros(U.num_params(), dtype=np.float32)
    sl = dict(U.layer_slices())
    b13 = np.zeros(16, dtype=np.float32)
    b13[0], b13[1], b13[2] = 1.0 + 2.0 ** -10, 3.0 + 2.0 ** -7, -5.0
    p[sl["b13"]] = b13
    hw = np.zeros(16, dtype=np.float32)
    hw[0], hw[1], hw[2] = 2.0, -0.5, 7.0
    p[sl["head"]] = np.concatenate([hw, [0.25]])
    smp = np.random.default_rng(5).standard_normal(3 * 8 ** 3)
    y64, t64 = U.predict(p, smp, 1.0, terms=True)
    yb, tb = U.predict(p, smp, 1.0, store=U.bf16_acts, terms=True)
    exact = 2.0 * (1.0 + 2.0 ** -10) - 0.5 * (3.0 + 2.0 ** -7) + 0.25
    assert np.allclose(y64, exact, rtol=0, atol=1e-12)
    assert np.all(yb == 2.0 * 1.0 - 0.5 * 3.0 + 0.25)
    assert np.all(tb == 2.0 * 1.0 + 0.5 * 3.0)
    assert np.allclose(t64, 2.0 * (1.0 + 2.0 ** -10) + 0.5 * (3.0 + 2.0 ** -7), rtol=0, atol=1e-12)


def test_bf16_activation_storage_stays_within_the_rounding_model():
    # storing activations in BF16 (relative rounding <= 2^-8 per value) moves a
    # random network's output by about a percent, never by more than a few
    rng = np.random.default_rng(6)
    p = he_params(6)
    S = 16
    smp = np.concatenate([rng.random(S ** 3), rng.standard_normal(S ** 3), rng.standard_normal(S ** 3)])
    y64 = U.predict(p, smp, 0.0)
    yb = U.predict(p, smp, 0.0, store=U.bf16_acts)
    rel = np.linalg.norm(yb - y64) / np.linalg.norm(y64)
    assert 1e-4 < rel < 3e-2
