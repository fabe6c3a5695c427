"""Pins of the oracle's mapping-side functions: the occupancy update (density at the 64^3 cell centres, moving
maximum, threshold) by closed forms, the full forward and brute-force bit layout; the Eq. 5 data-update angle by
closed forms."""
import numpy as np
import pytest

from oracle import romap_oracle as O


def test_cell_centres_closed_form_and_lookup():
    half = np.array([0.5, 0.37, 0.81], np.float32)
    rng = np.random.default_rng(0)
    for _ in range(200):
        i = rng.integers(0, 64, 3)
        x = O.cell_centre(half, *i)
        exact = -half.astype(np.float64) + (i + 0.5) * (2 * half.astype(np.float64) / 64)
        # two FP32 roundings (the product and the sum), each within one ulp of the box half-size
        assert np.all(np.abs(x - exact) <= 2 * np.spacing(half))
        # a grid with only this cell set: the lookup finds it at the centre and not at the neighbours' centres
        bits = np.zeros(4096, np.uint64)
        cell = int(i[0] + 64 * i[1] + 4096 * i[2])
        bits[cell >> 6] = np.uint64(1) << np.uint64(cell & 63)
        assert O.occupied(bits, x, half)
        for a in range(3):
            j = i.copy()
            j[a] = (j[a] + 1) % 64
            assert not O.occupied(bits, O.cell_centre(half, *j), half)
    # the unit box: centres are dyadic, hence exact
    assert np.array_equal(O.cell_centre(np.full(3, 0.5, np.float32), 0, 31, 63),
                          np.array([0.5 / 64 - 0.5, 31.5 / 64 - 0.5, 63.5 / 64 - 0.5], np.float32))


def _affine_model(A, b):
    """One dense level (N = 8, F = 2) filled with an affine field of vertex position; the first layer's unit 0 copies
    feature 0 and output 0 of the second layer copies unit 0: sigma = exp(clamp(relu(A x + b)))."""
    cfg = O.make_config(L=1, F=2, T=2 ** 12, n_min=8, growth=2.0, dir_dims=3)
    nh = O.hash_param_count(cfg)
    p = np.zeros(O.param_count(cfg))
    N = int(cfg.res[0])
    for z in range(N + 1):
        for y in range(N + 1):
            for x in range(N + 1):
                pos = np.array([x, y, z]) / N - 0.5
                p[O.grid_index(cfg, 0, x, y, z) * 2] = A @ pos + b
    W0 = nh + O.mlp_layer_offset(cfg, 0)
    W1 = nh + O.mlp_layer_offset(cfg, 1)
    p[W0 + 0] = 1.0          # W0[0][0]: unit 0 <- feature 0
    p[W1 + 0] = 1.0          # W1[0][0]: output 0 <- unit 0
    return cfg, p


def test_density_closed_form():
    half = np.full(3, 0.5, np.float32)
    A, b = np.array([3.0, -2.0, 1.5]), 0.4
    cfg, p = _affine_model(A, b)
    rng = np.random.default_rng(1)
    for _ in range(100):
        i = rng.integers(0, 64, 3)
        x = O.cell_centre(half, *i)
        want = np.exp(min(max(A @ x.astype(np.float64) + b, 0.0), 15.0))
        assert O.density(cfg, p, x, half) == pytest.approx(want, rel=1e-12)
    # zero table: sigma = exp(0) = 1 everywhere
    cfg2 = O.make_config(L=4, T=2 ** 10, growth=2.0)
    p2 = O.init_params(cfg2, 5)
    p2[:O.hash_param_count(cfg2)] = 0.0
    assert np.all(O.density_grid(cfg2, p2, half) == 1.0)
    # clamp at 15
    cfg3, p3 = _affine_model(np.zeros(3), 40.0)
    assert O.density(cfg3, p3, np.zeros(3, np.float32), half) == pytest.approx(np.exp(15.0), rel=1e-14)


def test_density_matches_full_forward():
    """The density-only evaluation equals sigma of the full two-net forward (pinned against numpy GEMMs)."""
    cfg = O.make_config(L=8, T=2 ** 12, growth=1.5)
    rng = np.random.default_rng(2)
    p = O.init_params(cfg, 9)
    nh = O.hash_param_count(cfg)
    p[:nh] = rng.uniform(-1, 1, nh)
    half = np.array([0.4, 0.5, 0.3], np.float32)
    for _ in range(20):
        x = (rng.uniform(-1, 1, 3) * half).astype(np.float32)
        enc = O.encode(cfg, p[:nh], x, half)
        f = O.mlp_forward(cfg, p[nh:], enc, np.array([0.0, 0.0, 1.0], np.float32))
        assert O.density(cfg, p, x, half) == pytest.approx(f["sigma"], rel=1e-13)


def test_moving_maximum_and_bits_brute_force():
    rng = np.random.default_rng(3)
    n = 64 ** 3
    d0 = rng.exponential(1.0, n)
    s = rng.exponential(1.0, n)
    decay, thr = 0.95, 0.8
    d1, bits = O.occupancy_update(s, decay, thr, d0)
    assert np.array_equal(d1, np.maximum(decay * d0, s))
    want = np.zeros(4096, np.uint64)
    for i in np.nonzero(d1 > thr)[0]:
        want[i >> 6] |= np.uint64(1) << np.uint64(i & 63)
    assert np.array_equal(bits, want)
    # the bits drive the sampler's occupancy lookup at the cell centres
    half = np.array([0.5, 0.5, 0.5], np.float32)
    for _ in range(300):
        i = rng.integers(0, 64, 3)
        cell = int(i[0] + 64 * i[1] + 4096 * i[2])
        assert O.occupied(bits, O.cell_centre(half, *i), half) == (d1[cell] > thr)
    # decay 0: the new density replaces the old one; repeated updates with the same sigma are idempotent
    d2, b2 = O.occupancy_update(s, 0.0, thr, d1)
    assert np.array_equal(d2, s)
    d3, b3 = O.occupancy_update(s, 0.0, thr, d2)
    assert np.array_equal(d3, d2) and np.array_equal(b3, b2)


def test_view_angle_closed_forms():
    """Eq. 5 against closed forms: orthogonal, coincident and opposite directions, a 25-degree rotation about an
    arbitrary object centre (scale-free in the distances), and the first image always updating."""
    o = np.array([0.3, -1.2, 0.8])
    assert O.view_angle_deg(o + [1, 0, 0], o + [0, 3, 0], o) == pytest.approx(90.0, abs=1e-12)
    assert O.view_angle_deg(o + [1, 2, 3], o + [2, 4, 6], o) == pytest.approx(0.0, abs=1e-6)
    assert O.view_angle_deg(o + [1, 2, 3], o - [2, 4, 6], o) == pytest.approx(180.0, abs=1e-6)
    rng = np.random.default_rng(4)
    for deg in (5.0, 24.9, 25.1, 60.0, 133.0):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        v = np.cross(axis, rng.normal(size=3))
        v /= np.linalg.norm(v)
        th = np.deg2rad(deg)
        w = v * np.cos(th) + np.cross(axis, v) * np.sin(th)  # v rotated about axis (axis _|_ v)
        got = O.view_angle_deg(o + 2.5 * v, o + 0.7 * w, o)
        assert got == pytest.approx(deg, abs=1e-9)
        assert O.should_update(o + 2.5 * v, o + 0.7 * w, o, 25.0) == (deg > 25.0)
    assert O.should_update(None, o + [1, 0, 0], o, 25.0)
    assert O.view_angle_deg(o, o + [1, 0, 0], o) == 180.0  # degenerate: a camera at the object centre


def test_lattice_and_crossing_vertices_closed_forms():
    """Lattice vertices in closed form (the unit box is dyadic: exact); with an affine density field the crossing
    vertices lie exactly on the iso-plane and there is one per lattice edge the plane cuts."""
    half = np.full(3, 0.5, np.float32)
    assert np.array_equal(O.lattice_vertex(half, 0, 32, 64), np.array([-0.5, 0.0, 0.5], np.float32))
    h2 = np.array([0.3, 0.45, 0.7], np.float32)
    for i in (0, 1, 17, 63, 64):
        x = O.lattice_vertex(h2, i, 64 - i, i)
        exact = -h2.astype(np.float64) + np.array([i, 64 - i, i]) * (2 * h2.astype(np.float64) / 64)
        assert np.all(np.abs(x - exact) <= 2 * np.spacing(h2))
    # sigma = 2 + x + 2 y - z at the lattice vertices, iso 2.1: the plane x + 2y - z = 0.1
    g = np.array([O.lattice_vertex(half, i, j, k) for k in range(65) for j in range(65) for i in range(65)],
                 np.float64)
    sigma = 2.0 + g[:, 0] + 2.0 * g[:, 1] - g[:, 2]
    codes, pos = O.mesh_vertices(sigma, half, 2.1)
    assert np.allclose(pos[:, 0] + 2 * pos[:, 1] - pos[:, 2], 0.1, atol=1e-12)
    # brute force over all lattice edges
    want = []
    for v in range(65 ** 3):
        i, j, k = v % 65, (v // 65) % 65, v // 65 ** 2
        for d, (di, dj, dk) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            if (i, j, k)[d] == 64:
                continue
            u = (i + di) + 65 * (j + dj) + 65 ** 2 * (k + dk)
            if (sigma[v] > 2.1) != (sigma[u] > 2.1):
                want.append(3 * v + d)
    assert np.array_equal(codes, np.array(want, np.int64))
