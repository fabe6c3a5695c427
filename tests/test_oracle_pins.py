"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks one part of the oracle against a closed form, an invariant,
a brute-force enumeration, a library routine (numpy GEMM, torch autograd,
torch.optim.Adam) or central finite differences, chosen so that a plausible
mistake (dropped term, wrong sign or index, transposed operand) fails.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import romap_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# Random numbers (reading R-1): Philox4x32-10 known answers
# ----------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if ln.strip() and ln[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_u01_exact_range_and_moments():
    assert O.u01(0) == 0.0
    assert O.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert O.u01(0x80000000) == 0.5
    xs = [O.philox([i, 7, 3, 0], [11, 13]) for i in range(4000)]
    u = np.array([O.u01(int(w)) for x in xs for w in x])
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005


# ----------------------------------------------------------------------------
# Grid layout (readings R-4, R-5)
# ----------------------------------------------------------------------------
def _icbrt(n):
    r = int(round(n ** (1 / 3)))
    while r ** 3 > n:
        r -= 1
    while (r + 1) ** 3 <= n:
        r += 1
    return r


def test_level_resolutions_geometric_exact():
    # 16 -> 512 over 16 levels: b = 2^(1/3), N_l = floor(16 * 2^(l/3)) = floor(cbrt(16^3 * 2^l)).
    res = O.level_resolutions(16, 16, 0.0, 512)
    exact = [_icbrt(16 ** 3 * 2 ** l) for l in range(16)]
    assert list(res) == exact
    # growth 1.5 over 8 levels: N_l = floor(16 * (3/2)^l) in exact rational arithmetic.
    res = O.level_resolutions(8, 16, 1.5)
    exact = [math.floor(Fraction(16) * Fraction(3, 2) ** l) for l in range(8)]
    assert list(res) == exact
    # L=4, b=2: 16, 32, 64, 128
    assert list(O.level_resolutions(4, 16, 2.0)) == [16, 32, 64, 128]


def test_param_counts_by_enumeration():
    cfg = O.make_config(L=16, T=2 ** 16, n_min=16, growth=0.0, n_max=512)
    res = O.level_resolutions(16, 16, 0.0, 512)
    sizes = [min((n + 1) ** 3, 2 ** 16) for n in res]
    assert 2 * sum(sizes) == 1708238  # live entries; each level's storage starts at a multiple of 8 entries
    padded = [(n + 7) // 8 * 8 for n in sizes]
    assert O.hash_param_count(cfg) == 2 * sum(padded) == 1708272
    assert O.param_count(cfg) - O.hash_param_count(cfg) == 64 * 32 + 16 * 64 + 64 * 18 + 64 * 64 + 3 * 64
    for l in range(16):
        assert O.level_offset(cfg, l) == sum(padded[:l])
        assert O.level_is_dense(cfg, l) == ((res[l] + 1) ** 3 <= 2 ** 16)


def test_dense_level_is_a_bijection():
    cfg = O.make_config(L=2, T=2 ** 12, n_min=6, growth=2.0)  # N = 6 (343 dense), 12 (2197 dense)
    for l in range(2):
        n = int(cfg.res[l]) + 1
        assert O.level_is_dense(cfg, l)
        seen = sorted(O.grid_index(cfg, l, x, y, z) for z in range(n) for y in range(n) for x in range(n))
        assert seen == list(range(n ** 3))


def test_spatial_hash_definition():
    # Mueller et al. 2022, Eq. 4: h(x) = (xor_i x_i pi_i) mod T, pi = (1, 2654435761, 805459861).
    cfg = O.make_config(L=2, T=2 ** 10, n_min=16, growth=2.0)
    assert not O.level_is_dense(cfg, 0)
    T = 2 ** 10
    for x in range(0, 40):
        assert O.grid_index(cfg, 0, x, 0, 0) == x % T        # pi_1 = 1
    assert O.grid_index(cfg, 0, 0, 1, 0) == 2654435761 % T
    assert O.grid_index(cfg, 0, 0, 0, 1) == 805459861 % T
    assert O.grid_index(cfg, 0, 1, 1, 0) == (1 ^ 2654435761) % T  # xor, not +
    assert O.grid_index(cfg, 0, 3, 5, 7) == (3 ^ (5 * 2654435761 % 2 ** 32) ^ (7 * 805459861 % 2 ** 32)) % T


def test_corners_match_brute_force_enumeration():
    """For random points, the 8 (index, weight) pairs equal those found by enumerating every vertex of the
    level and keeping those within one cell of the point, with tent weights prod(1 - |v - p|)."""
    cfg = O.make_config(L=3, T=2 ** 8, n_min=5, growth=1.5)   # N = 5 (216 dense), 7 (512 hashed), 11 (hashed)
    half = np.array([0.5, 0.4, 0.3], np.float32)
    rng = np.random.default_rng(3)
    for l in range(3):
        N = int(cfg.res[l])
        verts = np.array([(x, y, z) for z in range(N + 1) for y in range(N + 1) for x in range(N + 1)])
        vidx = np.array([O.grid_index(cfg, l, *map(int, v)) for v in verts])
        for _ in range(25):
            x = (rng.uniform(-1, 1, 3) * half * 0.999).astype(np.float32)
            idx, w = O.level_corners(cfg, l, x, half)
            p = (x.astype(np.float64) + half) / (2 * half) * N
            near = np.all(np.abs(verts - p) < 1.0, axis=1)
            tent = np.prod(1.0 - np.abs(verts[near] - p), axis=1)
            ref = {}
            for i, t in zip(vidx[near], tent):
                ref[int(i)] = ref.get(int(i), 0.0) + t
            got = {}
            for i, t in zip(idx, w):
                got[int(i)] = got.get(int(i), 0.0) + t
            assert set(ref) == set(got)
            for k in ref:
                assert abs(ref[k] - got[k]) < 1e-5
            assert abs(sum(w) - 1.0) < 1e-12


def test_encoding_reproduces_affine_field():
    """Dense levels filled with an affine function of vertex position reproduce it exactly (trilinear
    interpolation is exact on affine fields): pins weights, dense indexing, level offsets, feature order."""
    cfg = O.make_config(L=2, F=2, T=2 ** 12, n_min=6, growth=2.0)
    half = np.array([0.5, 0.5, 0.5], np.float32)
    table = np.zeros(O.hash_param_count(cfg))
    A = np.array([[0.3, -1.2, 0.7], [2.0, 0.1, -0.4]])
    b = np.array([0.25, -0.5])
    for l in range(2):
        N = int(cfg.res[l])
        off = O.level_offset(cfg, l)
        for z in range(N + 1):
            for y in range(N + 1):
                for x in range(N + 1):
                    pos = np.array([x, y, z]) / N * 1.0 - 0.5
                    i = O.grid_index(cfg, l, x, y, z)
                    for k in range(2):
                        table[(off + i) * 2 + k] = A[k] @ pos + b[k] + 10 * l
    rng = np.random.default_rng(0)
    for _ in range(50):
        x = rng.uniform(-0.5, 0.5, 3).astype(np.float32)
        enc = O.encode(cfg, table, x, half)
        for l in range(2):
            N = int(cfg.res[l])
            # the point's grid coordinate as the oracle forms it (FP32), then the affine field
            u = np.clip((x - np.float32(-0.5)) * np.float32(1.0), 0, 1).astype(np.float32)
            pos = (u.astype(np.float32) * np.float32(N)).astype(np.float64) / N - 0.5
            for k in range(2):
                assert abs(enc[2 * l + k] - (A[k] @ pos + b[k] + 10 * l)) < 1e-12


# ----------------------------------------------------------------------------
# Sampler stage (readings R-2, R-3, R-7, R-8)
# ----------------------------------------------------------------------------
def _analytic_slab(o, d, half):
    o, d = o.astype(np.float64), d.astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        ta, tb = (-half - o) / d, (half - o) / d
    t0 = np.nanmax(np.minimum(ta, tb))
    t1 = np.nanmin(np.maximum(ta, tb))
    return max(t0, 0.0), t1


def test_slab_and_stratified_samples():
    rng = np.random.default_rng(5)
    half = np.array([0.5, 0.3, 0.4], np.float32)
    N = 32
    n_hit = 0
    for r in range(300):
        o = (rng.normal(size=3) * 1.5).astype(np.float32)
        d = rng.uniform(-0.6, 0.6, 3) - o if r % 4 else rng.normal(size=3)   # mostly aimed at the box
        d = (d / np.linalg.norm(d)).astype(np.float32)
        s = O.sample_ray(o, d, half, N, seed=9, step=3, slot=r, jitter=True)
        tn, tf = _analytic_slab(o, d, half.astype(np.float64))
        if not s["hit"]:
            assert not (tf > tn + 1e-5)
            assert not s["live"].any()
            continue
        n_hit += 1
        assert abs(s["t_near"] - tn) < 1e-5 and abs(s["t_far"] - tf) < 1e-5
        t = s["t"].astype(np.float64)
        step_len = (s["t_far"] - s["t_near"]) / N
        i = np.arange(N)
        # stratification: t_i in [t_near + i*dt, t_near + (i+1)*dt]
        assert np.all(t >= s["t_near"] + i * step_len - 1e-5) and np.all(t <= s["t_near"] + (i + 1) * step_len + 1e-5)
        assert np.all(np.diff(t) >= 0)
        assert abs(s["delta"].astype(np.float64).sum() - (s["t_far"] - t[0])) < 1e-5
        assert np.allclose(s["x"], o.astype(np.float64) + t[:, None] * d.astype(np.float64), atol=1e-5)
        assert np.all(np.abs(s["x"]) <= half + 1e-5)
    assert n_hit > 120


def test_midpoint_samples_without_jitter():
    o = np.array([0.0, 0.0, -2.0], np.float32)
    d = np.array([0.0, 0.0, 1.0], np.float32)
    half = np.array([0.5, 0.5, 0.5], np.float32)
    s = O.sample_ray(o, d, half, 8, seed=0, step=1, slot=0, jitter=False)
    assert s["hit"] and s["t_near"] == 1.5 and s["t_far"] == 2.5
    assert np.allclose(s["t"], 1.5 + (np.arange(8) + 0.5) / 8, atol=1e-7)
    assert np.allclose(s["delta"], [0.125] * 7 + [0.0625], atol=1e-7)


def test_ray_inside_box_and_axis_parallel():
    half = np.array([0.5, 0.5, 0.5], np.float32)
    hit, tn, tf = O.ray_aabb(np.zeros(3), np.array([1.0, 0.0, 0.0]), half)   # starts inside, d_y = d_z = 0
    assert hit and tn == 0.0 and tf == 0.5
    hit, _, _ = O.ray_aabb(np.array([0.0, 0.7, -2.0]), np.array([0.0, 0.0, 1.0]), half)  # parallel, outside y slab
    assert not hit
    hit, _, _ = O.ray_aabb(np.array([0.0, 0.0, 2.0]), np.array([0.0, 0.0, 1.0]), half)   # pointing away
    assert not hit


def test_world_to_object_matches_rotation_matrix():
    rng = np.random.default_rng(1)
    o = rng.normal(size=(50, 3))
    d = rng.normal(size=(50, 3)) * 3.0
    t = np.array([0.3, -1.2, 0.5])
    for yaw in (0.0, 0.7, -2.9):
        oo, do = O.world_to_object(o, d, t, yaw)
        c, s = math.cos(yaw), math.sin(yaw)
        R = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
        ref_o = (o.astype(np.float32).astype(np.float64) - t) @ R           # R^T (x - t)
        ref_d = d.astype(np.float32).astype(np.float64) @ R
        ref_d /= np.linalg.norm(ref_d, axis=1, keepdims=True)
        assert np.allclose(oo.reshape(-1, 3), ref_o, atol=2e-6)
        assert np.allclose(do.reshape(-1, 3), ref_d, atol=2e-7)


def test_occupancy_cells_brute_force():
    rng = np.random.default_rng(2)
    bits = rng.integers(0, 2 ** 63, size=4096, dtype=np.uint64) | (rng.integers(0, 2, size=4096, dtype=np.uint64) << np.uint64(63))
    flat = np.array([(int(bits[i >> 6]) >> (i & 63)) & 1 for i in range(64 ** 3)], np.uint8).reshape(64, 64, 64)
    half = np.array([0.5, 0.25, 1.0], np.float32)
    for _ in range(400):
        x = (rng.uniform(-1, 1, 3) * half).astype(np.float32)
        cell = np.floor((x.astype(np.float64) + half) / (2 * half) * 64).astype(int)
        if np.any(np.abs((x.astype(np.float64) + half) / (2 * half) * 64 - np.round((x + half) / (2 * half) * 64)) < 1e-4):
            continue
        cell = np.clip(cell, 0, 63)
        assert O.occupied(bits, x, half) == bool(flat[cell[2], cell[1], cell[0]])
    assert O.occupied(None, np.zeros(3), half)


# ----------------------------------------------------------------------------
# Volume rendering (Eq. 6) and its adjoint (reading R-10)
# ----------------------------------------------------------------------------
def test_composite_constant_density_closed_form():
    rng = np.random.default_rng(0)
    for _ in range(20):
        n = int(rng.integers(1, 40))
        sigma = float(rng.uniform(0.1, 30))
        delta = rng.uniform(0.001, 0.05, n)
        t = np.cumsum(delta)
        c = rng.uniform(0, 1, 3)
        bg = rng.uniform(0, 1, 3)
        out, w = O.composite(np.full(n, sigma), delta, t, np.tile(c, (n, 1)), bg)
        A = 1 - math.exp(-sigma * delta.sum())                 # ray opacity 1 - exp(-sigma * d)
        assert abs(out[4] - A) < 1e-12
        assert np.allclose(out[:3], c * A + bg * (1 - A), atol=1e-12)
        assert abs(w.sum() - A) < 1e-12 and w.sum() <= 1.0   # telescoping: sum w = 1 - T_{N+1} <= 1


def test_composite_depth_geometric_series():
    sigma, dlt, t0, n = 7.0, 0.03, 1.1, 25
    q = math.exp(-sigma * dlt)
    t = t0 + dlt * np.arange(n)
    out, _ = O.composite(np.full(n, sigma), np.full(n, dlt), t, np.zeros((n, 3)), np.zeros(3))
    s_iq = q * (1 - n * q ** (n - 1) + (n - 1) * q ** n) / (1 - q) ** 2   # sum_{i<n} i q^i
    ref = (1 - q) * (t0 * (1 - q ** n) / (1 - q) + dlt * s_iq)
    assert abs(out[3] - ref) < 1e-12


def test_composite_zero_density():
    n = 10
    out, w = O.composite(np.zeros(n), np.full(n, 0.1), np.arange(n) * 0.1, np.random.rand(n, 3), np.array([0.2, 0.3, 0.4]))
    assert np.allclose(out[:3], [0.2, 0.3, 0.4]) and out[3] == 0.0 and out[4] == 0.0 and np.all(w == 0)


def test_composite_single_sample_gradient_closed_form():
    sigma, dlt, t = 3.0, 0.2, 1.4
    c, bg = np.array([0.9, 0.1, 0.4]), np.array([0.3, 0.6, 0.2])
    gC = np.array([1.0, -2.0, 0.5])
    gs, gc = O.composite_backward([sigma], [dlt], [t], c[None], bg, gC, 0.7, -0.3)
    e = math.exp(-sigma * dlt)
    ref = dlt * e * (gC @ (c - bg)) + 0.7 * dlt * e * t + (-0.3) * dlt * e
    assert abs(gs[0] - ref) < 1e-12
    assert np.allclose(gc[0], gC * (1 - e), atol=1e-15)


def test_composite_adjoint_matches_finite_differences():
    rng = np.random.default_rng(4)
    n = 23
    sigma = rng.uniform(0, 20, n)
    delta = rng.uniform(0.001, 0.08, n)
    t = 0.5 + np.cumsum(delta)
    c = rng.uniform(0, 1, (n, 3))
    bg = rng.uniform(0, 1, 3)
    gC, gD, gA = rng.normal(size=3), 0.37, -0.81

    def f(s, cc):
        out, _ = O.composite(s, delta, t, cc, bg)
        return gC @ out[:3] + gD * out[3] + gA * out[4]

    gs, gc = O.composite_backward(sigma, delta, t, c, bg, gC, gD, gA)
    h = 1e-6
    for i in range(n):
        e = np.zeros(n); e[i] = h
        fd = (f(sigma + e, c) - f(sigma - e, c)) / (2 * h)
        assert abs(fd - gs[i]) < 1e-7 * max(1, abs(fd))
        for k in range(3):
            E = np.zeros((n, 3)); E[i, k] = h
            fd = (f(sigma, c + E) - f(sigma, c - E)) / (2 * h)
            assert abs(fd - gc[i, k]) < 1e-7


# ----------------------------------------------------------------------------
# MLP (reading R-11, R-13): library GEMM and library autodiff
# ----------------------------------------------------------------------------
def _mlp_weights(cfg, mlp):
    shapes = [(cfg.hidden, cfg.L * cfg.F), (1 + cfg.geo, cfg.hidden), (cfg.hidden, cfg.geo + cfg.dir_dims),
              (cfg.hidden, cfg.hidden), (3, cfg.hidden)]
    if cfg.single_net:
        shapes += [(cfg.hidden, cfg.hidden)] * (cfg.hidden_layers - 1)
    Ws, off = [], 0
    for (o, i) in shapes:
        Ws.append(mlp[off:off + o * i].reshape(o, i))
        off += o * i
    return Ws


def test_mlp_forward_equals_matrix_products():
    cfg = O.make_config(L=16, T=2 ** 16, n_min=16, growth=0.0, n_max=512)
    rng = np.random.default_rng(0)
    nm = O.param_count(cfg) - O.hash_param_count(cfg)
    mlp = rng.normal(size=nm) * 0.3
    W = _mlp_weights(cfg, mlp)
    for _ in range(10):
        enc = rng.normal(size=32)
        dr = rng.normal(size=3).astype(np.float32)
        f = O.mlp_forward(cfg, mlp, enc, dr)
        h1 = np.maximum(W[0] @ enc, 0)
        out = W[1] @ h1
        h2 = np.maximum(W[2] @ np.concatenate([out[1:], dr.astype(np.float64)]), 0)
        h3 = np.maximum(W[3] @ h2, 0)
        logit = W[4] @ h3
        assert np.allclose(f["out"], out, rtol=1e-13, atol=1e-13)
        assert np.allclose(f["rgb"], 1 / (1 + np.exp(-logit)), rtol=1e-13)
        assert abs(f["sigma"] - math.exp(min(max(out[0], -15), 15))) < 1e-12 * f["sigma"]


def test_mlp_backward_equals_torch_autograd():
    torch = pytest.importorskip("torch")
    cfg = O.make_config(L=8, T=2 ** 12)
    rng = np.random.default_rng(1)
    nm = O.param_count(cfg) - O.hash_param_count(cfg)
    mlp = rng.normal(size=nm) * 0.3
    for trial in range(5):
        enc = rng.normal(size=16)
        dr = rng.normal(size=3).astype(np.float32)
        gsig, grgb = rng.normal(), rng.normal(size=3)
        f = O.mlp_forward(cfg, mlp, enc, dr)
        gmlp, genc = O.mlp_backward(cfg, mlp, f, gsig, grgb)
        tm = torch.tensor(mlp, dtype=torch.float64, requires_grad=True)
        te = torch.tensor(enc, dtype=torch.float64, requires_grad=True)
        Ws = _mlp_weights(cfg, tm)
        h1 = torch.relu(Ws[0] @ te)
        out = Ws[1] @ h1
        sigma = torch.exp(torch.clamp(out[0], -15, 15))
        h2 = torch.relu(Ws[2] @ torch.cat([out[1:], torch.tensor(dr, dtype=torch.float64)]))
        h3 = torch.relu(Ws[3] @ h2)
        rgb = torch.sigmoid(Ws[4] @ h3)
        (gsig * sigma + (torch.tensor(grgb) * rgb).sum()).backward()
        assert np.allclose(gmlp, tm.grad.numpy(), rtol=1e-11, atol=1e-12)
        assert np.allclose(genc, te.grad.numpy(), rtol=1e-11, atol=1e-12)


# ----------------------------------------------------------------------------
# Adam (reading R-14): closed form of the first step, torch.optim.Adam
# ----------------------------------------------------------------------------
def test_adam_first_step_moves_by_lr_sign():
    rng = np.random.default_rng(0)
    n = 1000
    p = rng.normal(size=n)
    g = rng.normal(size=n) * 10.0 ** rng.uniform(-6, 2, n)
    g[::7] = 0.0
    p1, m, v = O.adam(p, np.zeros(n), np.zeros(n), g, 1, 1e-2, 0.9, 0.99, 1e-15)
    moved = p - p1
    nz = g != 0
    # step 1: m_hat = g, v_hat = g^2, so the move is lr * g / (|g| + eps) = lr * sign(g) up to eps/|g|
    assert np.allclose(moved[nz], 1e-2 * g[nz] / (np.abs(g[nz]) + 1e-15), rtol=0, atol=1e-13)
    big = np.abs(g) > 1e-2
    assert np.allclose(moved[big], 1e-2 * np.sign(g[big]), rtol=0, atol=1e-13)
    assert np.all(moved[g == 0] == 0.0)


def test_adam_matches_torch_optim():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    n = 257
    p = rng.normal(size=n)
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=3e-3, betas=(0.9, 0.99), eps=1e-8)
    m = np.zeros(n); v = np.zeros(n)
    for step in range(1, 6):
        g = rng.normal(size=n)
        p, m, v = O.adam(p, m, v, g, step, 3e-3, 0.9, 0.99, 1e-8)
        tp.grad = torch.tensor(g)
        opt.step()
        assert np.allclose(p, tp.detach().numpy(), rtol=0, atol=1e-14)


# ----------------------------------------------------------------------------
# Parameter init (R-6, R-13) and batch draw (R-1)
# ----------------------------------------------------------------------------
def test_init_params_ranges_and_moments():
    cfg = O.make_config(L=16, T=2 ** 16, n_min=16, growth=0.0, n_max=512)
    p = O.init_params(cfg, 12345)
    nh = O.hash_param_count(cfg)
    h = p[:nh]
    assert np.all(np.abs(h) <= 1e-4) and abs(h.mean()) < 1e-6 and abs(h.var() - 1e-8 / 3) < 1e-10
    for layer, (o, i) in enumerate([(64, 32), (16, 64), (64, 18), (64, 64), (3, 64)]):
        off = nh + O.mlp_layer_offset(cfg, layer)
        w = p[off:off + o * i]
        lim = math.sqrt(6 / (o + i))
        assert np.all(np.abs(w) <= lim * (1 + 1e-6))
        assert abs(w.var() - lim ** 2 / 3) < 0.25 * lim ** 2 / 3
    assert not np.array_equal(p, O.init_params(cfg, 12346))


def test_draw_batch_in_order_and_uniform():
    cfg = O.make_config(rays_per_step=256, bg_random=False)
    idx, bg = O.draw_batch(cfg, 0, 1, 200)
    assert list(idx) == list(range(200)) and np.all(bg == 1.0)
    cfg = O.make_config(rays_per_step=4096, bg_random=True)
    idx, bg = O.draw_batch(cfg, 77, 3, 10)
    assert len(idx) == 10
    idx, bg = O.draw_batch(cfg, 77, 3, 10000)
    assert len(idx) == 4096 and idx.min() >= 0 and idx.max() < 10000
    counts = np.bincount(idx // 1000, minlength=10)
    assert np.all(np.abs(counts - 409.6) < 80)
    assert np.all((bg >= 0) & (bg < 1)) and abs(bg.mean() - 0.5) < 0.03
    idx2, _ = O.draw_batch(cfg, 77, 4, 10000)
    assert not np.array_equal(idx, idx2)


# ----------------------------------------------------------------------------
# Loss (Eq. 7-11, reading R-9) and the whole step
# ----------------------------------------------------------------------------
def _mixed_pool(n, rng, with_depth=True):
    o = np.zeros((n, 3)); d = np.zeros((n, 3))
    for r in range(n):
        az, el = rng.uniform(-np.pi, np.pi), rng.uniform(-0.5, 0.8)
        cam = 2.0 * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        tgt = rng.uniform(-0.3, 0.3, 3)
        dd = tgt - cam
        o[r], d[r] = cam, dd / np.linalg.norm(dd)
    cls = rng.integers(0, 3, n).astype(np.uint8)
    depth = np.full(n, np.nan)
    if with_depth:
        depth[::3] = rng.uniform(1.0, 3.0, len(depth[::3]))
    return dict(o=o.astype(np.float32), d=d.astype(np.float32), rgb=rng.uniform(0, 1, (n, 3)).astype(np.float32),
                depth=depth.astype(np.float32), cls=cls)


def test_zero_density_loss_invariant():
    """With every sample culled, sigma = 0: C_hat = b_r, so the R_b terms vanish and
    L = (1/B)[sum_{R_o} ||b_r - C||^2 + lambda1 sum_{R_d} |0 - D|]."""
    cfg = O.make_config(L=4, T=2 ** 10, growth=2.0, n_samples=16, rays_per_step=40, bg_random=True)
    rng = np.random.default_rng(0)
    pool = _mixed_pool(40, rng)
    p = O.init_params(cfg, 5)
    occ = np.zeros(4096, np.uint64)
    r = O.train_step(cfg, np.full(3, 0.5, np.float32), 5, 1, pool, p, np.zeros_like(p), np.zeros_like(p), occ=occ,
                     do_adam=False)
    bg = r["bg"]
    L = 0.0
    for i in range(40):
        if pool["cls"][i] == 2:
            continue
        if pool["cls"][i] == 0:
            L += np.sum((bg[i] - pool["rgb"][i].astype(np.float64)) ** 2)
        if np.isfinite(pool["depth"][i]):
            L += 0.5 * abs(float(pool["depth"][i]))
    assert abs(r["loss"][0] - L / 40) < 1e-12
    assert np.all(r["grad"][O.hash_param_count(cfg):] == 0)


def _constant_field_params(cfg, log_sigma):
    """Parameters whose model is a constant field: every hash entry 0.5, so every encoding feature is 0.5
    (trilinear weights sum to 1); density hidden unit 0 = relu(feature 0) = 0.5 and output 0 = 2 log_sigma * 0.5,
    so sigma = exp(log_sigma) everywhere; every other output, hence every colour-net input, hidden unit and logit,
    is 0, so the colour is sigmoid(0) = 1/2 in each channel, for every direction."""
    p = np.zeros(O.param_count(cfg))
    nh = O.hash_param_count(cfg)
    p[:nh] = 0.5
    LF = cfg.L * cfg.F
    p[nh + O.mlp_layer_offset(cfg, 0) + 0 * LF + 0] = 1.0      # W1[0][0] (layer 0 is H x LF, row-major)
    p[nh + O.mlp_layer_offset(cfg, 1) + 0 * cfg.hidden + 0] = 2.0 * log_sigma  # W2[0][0] (layer 1 is 16 x H)
    return p


def _live_by_grid(x, occ, half):
    """Occupancy of sample positions from the bitgrid's definition: cell c = min(floor(u * 64), 63) per axis with
    u = clamp((x + a) / (2 a), 0, 1) in FP32, bit c_x + 64 c_y + 4096 c_z."""
    x = np.asarray(x, np.float32)
    h = np.asarray(half, np.float32)
    u = np.clip((x - (-h)) * (np.float32(1.0) / (h - (-h))), 0, 1).astype(np.float32)
    c = np.minimum((u * np.float32(64.0)).astype(np.int64), 63)
    bit = c[..., 0] + 64 * c[..., 1] + 4096 * c[..., 2]
    words = np.asarray(occ, np.uint64)
    return ((words[bit >> 6] >> (bit & 63).astype(np.uint64)) & np.uint64(1)).astype(bool)


@pytest.mark.parametrize("culled", [False, True])
def test_density_loss_closed_form_constant_field(culled):
    """Eq. 7-11 at constant density sigma > 0 and constant colour c = 1/2, on a mix of object, background,
    occluder and depth rays.  Per ray with live-sample spacings delta_i: A = 1 - exp(-sigma sum_live delta_i),
    C_hat = c A + b (1 - A), D_hat = sum_live (T_i - T_{i+1}) t_i with T_i = exp(-sigma sum_{live j < i} delta_j);
    L = (1/B)[sum_{R_o} ||C_hat - C||^2 + sum_{R_b} ||C_hat - b||^2 + lambda1 sum_{R_d} |D_hat - D|
    + lambda2 sum_{R_b} sigma n_live].  With culled=True the bitgrid empties the half-box x < 0, so part of most rays
    is culled (O-8: no density term and no opacity there).  The density term counts live samples of R_b rays only."""
    sigma0, lam1, lam2, n = 3.0, 0.5, 0.04, 60
    cfg = O.make_config(L=4, T=2 ** 10, growth=2.0, n_samples=16, rays_per_step=n, bg_random=True,
                        lambda1=lam1, lambda2=lam2)
    rng = np.random.default_rng(31)
    pool = _mixed_pool(n, rng)
    pool["cls"][:6] = [0, 1, 2, 0, 1, 1]           # every class present whatever the draw
    half = np.full(3, 0.5, np.float32)
    occ = None
    if culled:
        cells = np.zeros(64 ** 3, bool)
        cells.reshape(64, 64, 64)[:, :, 32:] = True   # index [z][y][x]: keep cells with x >= 32 (x >= 0)
        occ = np.packbits(cells.reshape(-1, 64)[:, ::-1], axis=1).view(">u8").reshape(-1).astype(np.uint64)
    p = _constant_field_params(cfg, math.log(sigma0))
    z = np.zeros_like(p)
    r = O.train_step(cfg, half, 9, 1, pool, p, z, z, occ=occ, do_adam=False, want_samples=True)
    S = r["samples"]                                   # per sample: t, delta, x, y, z, live, sigma, dL/dsigma
    t, delta, x = S[..., 0], S[..., 1], S[..., 2:5]
    hit = np.array([O.ray_aabb(pool["o"][i], pool["d"][i], half)[0] for i in range(n)])
    live = hit[:, None] & (np.ones_like(t, bool) if occ is None else _live_by_grid(x, occ, half))
    bg = r["bg"]
    comps = np.zeros(4)
    n_culled = 0
    for i in range(n):
        dl = np.where(live[i], delta[i], 0.0)
        cum = np.concatenate([[0.0], np.cumsum(dl)])
        T = np.exp(-sigma0 * cum)
        A = 1.0 - T[-1]
        C_hat = 0.5 * A + bg[i] * (1.0 - A)
        D_hat = float(np.sum((T[:-1] - T[1:]) * t[i]))
        cls = pool["cls"][i]
        n_culled += int(hit[i]) * int(np.count_nonzero(~live[i]))
        if cls == 2:
            continue
        tgt = pool["rgb"][i].astype(np.float64) if cls == 0 else bg[i]
        comps[0 if cls == 0 else 1] += np.sum((C_hat - tgt) ** 2)
        if np.isfinite(pool["depth"][i]):
            comps[2] += abs(D_hat - float(pool["depth"][i]))
        if cls == 1:
            comps[3] += sigma0 * np.count_nonzero(live[i])
    L = (comps[0] + comps[1] + lam1 * comps[2] + lam2 * comps[3]) / n
    assert comps[3] > 0 and np.all(np.isfinite(comps))
    if culled:
        assert n_culled > 100                       # the grid really culls part of the rays
    assert abs(r["loss"][0] - L) < 1e-12, (r["loss"][0], L)
    assert np.allclose(r["loss"][1:], comps / n, rtol=0, atol=1e-12), (r["loss"][1:], comps / n)
    # the live flags and densities of the step agree with the bitgrid and the constant field
    assert np.array_equal(S[..., 5].astype(bool), live)
    assert np.allclose(S[..., 6][live], sigma0, rtol=1e-14) and np.all(S[..., 6][~live] == 0)


def _fd_check(cfg, params, pool, seed, step, occ, idx, h=1e-4, tol=1e-6):
    """Central differences of the step loss.  A parameter whose h=1e-4 difference disagrees is re-checked at
    h=1e-6: a ReLU or |.| kink within +-1e-4 of the point is the only legitimate cause of disagreement."""
    half = np.full(3, 0.5, np.float32)
    z = np.zeros_like(params)

    def loss(p):
        return O.train_step(cfg, half, seed, step, pool, p, z, z, occ=occ, do_adam=False)["loss"][0]

    g = O.train_step(cfg, half, seed, step, pool, params, z, z, occ=occ, do_adam=False)["grad"]
    scale = np.abs(g).max()
    worst, rechecked = 0.0, 0
    for i in idx:
        err = None
        for hh in (h, 1e-6):
            e = np.zeros_like(params); e[i] = hh
            fd = (loss(params + e) - loss(params - e)) / (2 * hh)
            err = abs(fd - g[i]) / scale
            if err < tol:
                break
            rechecked += 1
        worst = max(worst, err)
    assert worst < tol, worst
    assert rechecked <= max(2, len(idx) // 10), rechecked   # kinks are rare
    return g


def test_full_step_gradient_matches_finite_differences_small():
    """Every parameter of a tiny model (L=2, T=64, hidden 16), with all loss terms active."""
    cfg = O.make_config(L=2, T=64, n_min=4, growth=2.0, n_samples=8, rays_per_step=12, hidden=16, bg_random=True)
    rng = np.random.default_rng(7)
    pool = _mixed_pool(12, rng)
    params = rng.uniform(-1, 1, O.param_count(cfg)) * 0.5
    g = _fd_check(cfg, params, pool, 3, 2, None, range(O.param_count(cfg)))
    assert np.count_nonzero(g) > 0.5 * g.size


def test_step_gradient_matches_finite_differences_diffcheck_config():
    """Differentiation-check configuration: L=4, T=2^10 (16 -> 128, hash collisions), 64 rays x 16 samples;
    a sample of hash entries and MLP weights."""
    cfg = O.make_config(L=4, T=2 ** 10, n_min=16, growth=2.0, n_samples=16, rays_per_step=64, bg_random=True)
    rng = np.random.default_rng(11)
    pool = _mixed_pool(64, rng)
    params = O.init_params(cfg, 21)
    nh = O.hash_param_count(cfg)
    params[:nh] = rng.uniform(-1, 1, nh)         # non-trivial features
    base = O.train_step(cfg, np.full(3, 0.5, np.float32), 21, 1, pool, params, params * 0, params * 0, do_adam=False)
    touched = np.nonzero(base["grad"][:nh])[0]
    idx = list(rng.choice(touched, 40, replace=False)) + list(nh + rng.choice(O.param_count(cfg) - nh, 40, replace=False))
    _fd_check(cfg, params, pool, 21, 1, None, idx)


def test_train_step_equals_explicit_rays():
    """The step's loss and gradient equal those of the explicit-ray path on the drawn batch."""
    cfg = O.make_config(L=4, T=2 ** 10, growth=2.0, n_samples=16, rays_per_step=30, bg_random=True)
    rng = np.random.default_rng(2)
    pool = _mixed_pool(100, rng)
    p = O.init_params(cfg, 8)
    half = np.full(3, 0.5, np.float32)
    r = O.train_step(cfg, half, 8, 4, pool, p, p * 0, p * 0, do_adam=False, want_rays=True)
    i = r["pool_idx"]
    e = O.rays_loss_grad(cfg, p, half, 8, 4, pool["o"][i], pool["d"][i], pool["rgb"][i], pool["depth"][i],
                         pool["cls"][i], r["bg"], inv_B=1 / 30)
    assert abs(e["total"] / 30 - r["loss"][0]) < 1e-14
    assert np.array_equal(e["grad"], r["grad"])


def test_training_decreases_loss_config0():
    from paper_2304_05735_gb300 import synth
    sc = synth.config0_scene()
    cfg = O.make_config()   # L=8, T=2^12, 16 growth 1.5, 32 samples, 256 rays, white background
    o, d = O.world_to_object(sc.pool["origin"], sc.pool["dir"], sc.t, sc.yaw)
    pool = dict(o=o, d=d, rgb=sc.pool["rgb"], depth=sc.pool["depth"], cls=sc.pool["cls"])
    p = O.init_params(cfg, 0)
    m, v = np.zeros_like(p), np.zeros_like(p)
    losses = []
    half = sc.half.astype(np.float32)
    for step in range(1, 13):
        r = O.train_step(cfg, half, 0, step, pool, p, m, v)
        p, m, v = r["params"], r["m"], r["v"]
        losses.append(r["loss"][0])
    assert losses[-1] < 0.5 * losses[0]


@pytest.mark.parametrize("K", [1, 2, 3])
def test_single_net_forward_and_backward(K):
    """The paper's model (K hidden layers of 64, positions only; Table 4 times K = 1, 2, 3): sigma from output 0
    and the colour sigmoid(outputs 1..3) of the density net, against numpy matrix products and torch autograd; the
    colour-net weights get no gradient."""
    torch = pytest.importorskip("torch")
    cfg = O.make_config(L=8, T=2 ** 12, dir_dims=0, single_net=True, hidden_layers=K)
    rng = np.random.default_rng(3 + K)
    nm = O.param_count(cfg) - O.hash_param_count(cfg)
    assert nm == 64 * 16 + 16 * 64 + 64 * 15 + 64 * 64 + 3 * 64 + (K - 1) * 64 * 64
    mlp = rng.normal(size=nm) * 0.3
    W = _mlp_weights(cfg, mlp)
    for _ in range(5):
        enc = rng.normal(size=16)
        f = O.mlp_forward(cfg, mlp, enc, np.zeros(3, np.float32))
        h = np.maximum(W[0] @ enc, 0)
        for M in W[5:]:
            h = np.maximum(M @ h, 0)
        out = W[1] @ h
        assert np.allclose(f["rgb"], 1 / (1 + np.exp(-out[1:4])), rtol=1e-13)
        assert abs(f["sigma"] - math.exp(min(max(out[0], -15), 15))) < 1e-12 * f["sigma"]
        gsig, grgb = rng.normal(), rng.normal(size=3)
        gmlp, genc = O.mlp_backward(cfg, mlp, f, gsig, grgb)
        tm = torch.tensor(mlp, dtype=torch.float64, requires_grad=True)
        te = torch.tensor(enc, dtype=torch.float64, requires_grad=True)
        Ws = _mlp_weights(cfg, tm)
        th = torch.relu(Ws[0] @ te)
        for M in Ws[5:]:
            th = torch.relu(M @ th)
        o = Ws[1] @ th
        (gsig * torch.exp(torch.clamp(o[0], -15, 15)) + (torch.tensor(grgb) * torch.sigmoid(o[1:4])).sum()).backward()
        assert np.allclose(gmlp, tm.grad.numpy(), rtol=1e-11, atol=1e-12)
        assert np.allclose(genc, te.grad.numpy(), rtol=1e-11, atol=1e-12)
        off2, off5 = O.mlp_layer_offset(cfg, 2), O.mlp_layer_offset(cfg, 5)
        assert np.all(gmlp[off2:off5] == 0.0)
        if K > 1:
            assert np.any(gmlp[off5:] != 0.0)


def test_single_net_identity_hidden_layers_reduce_to_one():
    """Extra hidden layers equal to c I (c > 0) commute with ReLU: the K-layer network equals the one-layer network
    whose output layer is scaled by c^(K-1) in the rendered colour, the density (also through the occupancy-grid
    density) and the gradients of the encoding and the first layer; the output layer's gradient is c^(K-1) times
    the scaled network's."""
    cfg1 = O.make_config(L=8, T=2 ** 12, dir_dims=0, single_net=True, hidden_layers=1)
    rng = np.random.default_rng(17)
    p1 = O.init_params(cfg1, 2)
    nh = O.hash_param_count(cfg1)
    p1[:nh] = rng.uniform(-1, 1, nh)
    half = np.array([0.5, 0.4, 0.45], np.float32)
    for K, c in ((2, 1.0), (3, 0.7)):
        cfgK = O.make_config(L=8, T=2 ** 12, dir_dims=0, single_net=True, hidden_layers=K)
        pK = np.zeros(O.param_count(cfgK))
        pK[:p1.size] = p1
        offs = [nh + O.mlp_layer_offset(cfgK, 5 + k) for k in range(K - 1)]
        for o in offs:
            pK[o:o + 64 * 64] = (c * np.eye(64)).reshape(-1)
        pS = p1.copy()   # one layer, output layer scaled by c^(K-1)
        o1 = nh + O.mlp_layer_offset(cfg1, 1)
        pS[o1:o1 + 16 * 64] *= c ** (K - 1)
        enc = rng.normal(size=16)
        fK = O.mlp_forward(cfgK, pK[nh:], enc, np.zeros(3, np.float32))
        fS = O.mlp_forward(cfg1, pS[nh:], enc, np.zeros(3, np.float32))
        assert np.allclose(fK["rgb"], fS["rgb"], rtol=1e-13) and fK["sigma"] == pytest.approx(fS["sigma"], rel=1e-13)
        gK, eK = O.mlp_backward(cfgK, pK[nh:], fK, 0.3, np.array([0.1, -0.2, 0.4]))
        gS, eS = O.mlp_backward(cfg1, pS[nh:], fS, 0.3, np.array([0.1, -0.2, 0.4]))
        assert np.allclose(eK, eS, rtol=1e-12, atol=1e-15)
        n0 = 64 * 16
        assert np.allclose(gK[:n0], gS[:n0], rtol=1e-12, atol=1e-15)       # first layer
        assert np.allclose(gK[n0:n0 + 1024], gS[n0:n0 + 1024] * c ** (K - 1), rtol=1e-12, atol=1e-15)  # output
        x = rng.uniform(-0.4, 0.4, 3).astype(np.float32)
        assert O.density(cfgK, pK, x, half) == pytest.approx(O.density(cfg1, pS, x, half), rel=1e-13)