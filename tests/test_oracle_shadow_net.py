"""Pins of the oracle of the learned shadow-transmittance surrogate: spherical
harmonics, hash encoding, network, back-propagation, Adam and training pairs."""
import math

import numpy as np
import pytest

from paper_2309_04581_gb300 import scenes as S

TINY_T = 8   # 256 entries per level: levels with N <= 5 dense, the rest hashed
TINY_RES = [2, 3, 5, 7, 11, 16, 23, 32]


def _tiny_net(orc, seed=1, scale=0.3):
    # a table far from zero so that the hash features matter in the gradients
    p = S.snet_init(seed, log2_T=TINY_T, table_scale=scale).astype(np.float64)
    return orc.OracleShadowNet(TINY_RES, TINY_T, p)


def _sphere_quadrature(n_theta=24, n_phi=48):
    # Gauss-Legendre in cos(theta) x uniform in phi: exact for polynomials of degree < 2 n_theta
    x, wx = np.polynomial.legendre.leggauss(n_theta)
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    dirs, w = [], []
    for ct, wt in zip(x, wx):
        st = math.sqrt(1 - ct * ct)
        for ph in phi:
            dirs.append([st * math.cos(ph), st * math.sin(ph), ct])
            w.append(wt * 2 * math.pi / n_phi)
    return np.array(dirs), np.array(w)


def test_sh16_orthonormal_and_addition_theorem(orc):
    dirs, w = _sphere_quadrature()
    Y = np.array([orc.sh16(d) for d in dirs])
    gram = (Y * w[:, None]).T @ Y
    assert np.allclose(gram, np.eye(16), atol=1e-12)
    # each band l: sum_m Y_lm(w)^2 = (2l+1)/(4 pi) at every direction; parity (-1)^l
    rng = np.random.default_rng(0)
    for d in rng.normal(size=(20, 3)):
        d /= np.linalg.norm(d)
        y, yn = orc.sh16(d), orc.sh16(-d)
        for l in range(4):
            band = slice(l * l, (l + 1) * (l + 1))
            assert np.sum(y[band] ** 2) == pytest.approx((2 * l + 1) / (4 * math.pi), rel=1e-13)
            assert np.allclose(yn[band], (-1) ** l * y[band], atol=1e-15)


def test_encoding_reproduces_linear_tables_and_hashed_vertices(orc):
    net = _tiny_net(orc)
    T = 1 << TINY_T
    params = net.params.copy()
    # dense levels: table entries = a linear function of the vertex position ->
    # trilinear interpolation returns that function at any point inside the box
    for l, N in enumerate(TINY_RES):
        if (N + 1) ** 3 > T:
            continue
        for z in range(N + 1):
            for y in range(N + 1):
                for x in range(N + 1):
                    i = l * T + x + (N + 1) * (y + (N + 1) * z)
                    params[2 * i] = 0.3 * x / N - 0.7 * y / N + 0.2 * z / N
                    params[2 * i + 1] = 1.0 - x / N
    net2 = orc.OracleShadowNet(TINY_RES, TINY_T, params)
    rng = np.random.default_rng(3)
    for p in rng.uniform(-0.5, 0.5, (20, 3)):
        x = net2.encode(p, [0, 0, 1])
        u = p + 0.5
        for l, N in enumerate(TINY_RES):
            if (N + 1) ** 3 <= T:
                assert x[2 * l] == pytest.approx(0.3 * u[0] - 0.7 * u[1] + 0.2 * u[2], abs=1e-13)
                assert x[2 * l + 1] == pytest.approx(1.0 - u[0], abs=1e-13)
    # hashed levels at a grid vertex: exactly the entry at the spatial hash
    l, N = 6, TINY_RES[6]
    v = np.array([5, 17, 9])
    p = v / N - 0.5
    h = (int(v[0]) ^ (int(v[1]) * 2654435761 % 2**32) ^ (int(v[2]) * 805459861 % 2**32)) % T
    x = net.encode(p, [1, 0, 0])
    assert x[2 * l] == pytest.approx(net.params[2 * (l * T + h)], abs=1e-15)
    assert x[2 * l + 1] == pytest.approx(net.params[2 * (l * T + h) + 1], abs=1e-15)
    # the direction part is the spherical harmonics of the unit direction
    assert np.allclose(x[16:], orc.sh16(np.array([1.0, 0, 0])), atol=0)


def test_network_matches_torch_layers(orc):
    torch = pytest.importorskip("torch")
    net = _tiny_net(orc)
    T = 1 << TINY_T
    mlp = net.params[8 * T * 2:]
    W1 = mlp[:2048].reshape(64, 32); b1 = mlp[2048:2112]
    W2 = mlp[2112:6208].reshape(64, 64); b2 = mlp[6208:6272]
    W3 = mlp[6272:10368].reshape(64, 64); b3 = mlp[10368:10432]
    W4 = mlp[10432:10496].reshape(1, 64); b4 = mlp[10496:10497]
    rng = np.random.default_rng(4)
    for _ in range(10):
        p, w = rng.uniform(-0.5, 0.5, 3), rng.normal(size=3)
        x = torch.tensor(net.encode(p, w))
        F = torch.nn.functional
        h = F.relu(F.linear(x, torch.tensor(W1), torch.tensor(b1)))
        h = F.relu(F.linear(h, torch.tensor(W2), torch.tensor(b2)))
        h = F.relu(F.linear(h, torch.tensor(W3), torch.tensor(b3)))
        t = torch.sigmoid(F.linear(h, torch.tensor(W4), torch.tensor(b4)))
        assert net.forward(p, w) == pytest.approx(float(t), rel=1e-14)


def test_gradient_matches_central_differences(orc):
    net = _tiny_net(orc)
    rng = np.random.default_rng(5)
    m = 6
    pw = np.concatenate([rng.uniform(-0.45, 0.45, (m, 3)), rng.normal(size=(m, 3))], axis=1)
    y = rng.uniform(0, 1, m)
    loss, g = net.loss_grad(pw, y)
    T = 1 << TINY_T
    # every table entry the batch touches, plus a spread of network parameters
    touched = np.flatnonzero(g[:8 * T * 2] != 0)
    assert touched.size > 8 * 8   # corners on every level
    idx = np.concatenate([rng.choice(touched, 60, replace=False), 8 * T * 2 + rng.choice(10497, 120, replace=False),
                          [g.size - 1]])
    base = net.params.copy()
    for i in idx:
        h = 1e-6 * max(1.0, abs(base[i]))
        net.params[i] = base[i] + h
        lp, _ = net.loss_grad(pw, y, grad=False)
        net.params[i] = base[i] - h
        lm, _ = net.loss_grad(pw, y, grad=False)
        net.params[i] = base[i]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g).max(), 1e-12) + 1e-7 * abs(g[i]), (i, fd, g[i])
    assert loss == pytest.approx(np.mean([(net.forward(pw[k, :3], pw[k, 3:]) - y[k]) ** 2 for k in range(m)]),
                                 rel=1e-14)


def test_adam_matches_torch_and_constant_gradient_step(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    n = 50
    theta = rng.normal(size=n)
    m, v = np.zeros(n), np.zeros(n)
    tp = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.99), eps=1e-8)
    for t in range(1, 6):
        g = rng.normal(size=n)
        orc.adam_step(theta, m, v, g, t, 1e-2, 0.9, 0.99, 1e-8)
        tp.grad = torch.tensor(g)
        opt.step()
    assert np.allclose(theta, tp.detach().numpy(), rtol=1e-13, atol=1e-15)
    # a constant gradient moves every parameter by lr g / (|g| + eps) per step
    th, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    g = np.array([0.5, -2.0, 1e-3])
    for t in range(1, 4):
        before = th.copy()
        orc.adam_step(th, m, v, g, t, 0.1, 0.9, 0.99, 1e-15)
        assert np.allclose(th - before, -0.1 * g / (np.abs(g) + 1e-15), rtol=1e-12)


def test_training_pairs_follow_philox_and_the_march(orc):
    sc = S.config4(8, 8)
    seed, first, n = 11, 1000, 64
    pr = orc.shadow_pairs(sc, seed, first, n)
    key = (seed, 0x736861646F77)
    lo, hi = np.asarray(sc.field.aabb_min, np.float64), np.asarray(sc.field.aabb_max, np.float64)
    osc = orc.OracleScene(sc)
    for k in range(n):
        # numpy's Philox increments its counter before each block: start one below (first + k >= 1 here)
        bg = np.random.Philox(counter=np.array([first + k - 1, 0, 0, 0], np.uint64), key=np.array(key, np.uint64))
        u = (bg.random_raw(4) >> np.uint64(40)).astype(np.float64) / 2**24
        assert np.array_equal(pr[k, :3], lo + u[:3] * (hi - lo))
        l = min(int(u[3] * 4), 3)
        L = sc.lights[l]
        # the light point lies on the emitter triangle
        y = pr[k, :3] + pr[k, 3:6] * pr[k, 6]
        v0, v1, v2 = (np.asarray(x, np.float64) for x in (L.pos, L.v1, L.v2))
        A = np.column_stack([v1 - v0, v2 - v0])
        b, *_ = np.linalg.lstsq(A, y - v0, rcond=None)
        assert np.allclose(A @ b + v0, y, atol=1e-12) and b.min() >= -1e-12 and b.sum() <= 1 + 1e-12
        assert np.linalg.norm(pr[k, 3:6]) == pytest.approx(1.0, abs=1e-15)
        assert pr[k, 7] == orc.transmittance(osc, pr[k, :3], pr[k, 3:6], 0.0, pr[k, 6])
    assert 0.0 <= pr[:, 7].min() and pr[:, 7].max() <= 1.0
    assert pr[:, 7].min() < 0.5 < pr[:, 7].max()    # the field casts shadows on some pairs


def test_render_takes_shadow_transmittance_from_the_network(orc):
    # A network whose output is the constant sigmoid(b4) (all weights zero)
    # scales the next-event term of a point light by exactly that value, for
    # a shading point inside the field box; the march (sigma = 0.8) is not used.
    from tests.test_oracle_paths import _floor_scene, F
    p = np.zeros(S.snet_n_params(TINY_T))
    T_c = 0.3
    p[-1] = math.log(T_c / (1 - T_c))
    net = orc.OracleShadowNet(TINY_RES, TINY_T, p)
    x, z = 0.13, -0.07
    hp = np.array([F(x), F(-0.45), F(z)])
    lp = np.array([0.0, F(0.45), 0.0])
    D = np.linalg.norm(lp - hp)
    cos = (lp - hp)[1] / D
    sc = S.explicit_rays(_floor_scene(0.8), [[x, 0.3, z]], [[0, -1, 0]])
    t_cam = math.exp(-F(0.8) * (F(0.3) - F(-0.45)))
    got = orc.render(sc, shadow_net=net)["rgba"][0, :3]
    assert np.allclose(got, t_cam * 0.5 / math.pi * cos * 2.0 / D ** 2 * T_c, rtol=1e-12)
    marched = orc.render(sc)["rgba"][0, :3]
    assert np.allclose(marched, t_cam * 0.5 / math.pi * cos * 2.0 / D ** 2 * math.exp(-F(0.8) * D), rtol=1e-12)
