"""Mesh extraction (romap_extract_mesh, 64^3 marching cubes) against the oracle: lattice densities within FP32
tolerance; given the same lattice densities, the same crossed lattice edges in the same order and the same vertex
positions; a mesh whose every interior edge is shared by two oppositely oriented triangles, facing from the dense
side to the empty side; a closed sphere of Euler characteristic 2 at the right radius."""
import ctypes as C
import time

import numpy as np
import pytest

from oracle import romap_oracle as O
from paper_2304_05735_gb300 import romap as R

from _harness import Ctx, paired_config

pytestmark = pytest.mark.gpu


def _extract(ctx, oid, iso):
    nv, nt = C.c_int64(), C.c_int64()
    st = R.romap_extract_mesh(ctx.h, oid, iso, None, 0, None, 0, C.byref(nv), C.byref(nt), 0)
    assert st in (R.ROMAP_OK, R.ROMAP_ERR_CAPACITY)
    v = np.zeros((max(nv.value, 1), 3), np.float32)
    t = np.zeros((max(nt.value, 1), 3), np.int32)
    R.check(R.romap_extract_mesh(ctx.h, oid, iso, v.ctypes.data, nv.value, t.ctypes.data, nt.value, C.byref(nv),
                                 C.byref(nt), 0))
    return v[:nv.value], t[:nt.value]


def _lattice(ctx, oid):
    d = np.zeros(65 ** 3, np.float32)
    R.check(R.romap_density_lattice(ctx.h, oid, d.ctypes.data, 0))
    return d


def _edge_check(codes, tris, dens, iso):
    """Every directed mesh edge appears once; an undirected edge is shared by two triangles in opposite directions
    unless both of its vertices lie on one face of the box.  Returns the fraction of triangles facing outwards."""
    vi = codes // 3
    ax = codes % 3
    ijk = np.stack([vi % 65, (vi // 65) % 65, vi // 65 ** 2], 1)
    directed = {}
    for a, b, c in tris:
        for u, w in ((a, b), (b, c), (c, a)):
            assert (u, w) not in directed
            directed[(u, w)] = True
    for (u, w) in directed:
        if (w, u) in directed:
            continue
        on_face = False
        for axis in range(3):
            for side in (0, 64):
                if all(ijk[x, axis] == side and ax[x] != axis for x in (u, w)):
                    on_face = True
        assert on_face, (u, w)
    return directed


def _outward_fraction(verts, tris, codes, dens, iso):
    vi, ax = codes // 3, codes % 3
    step = np.array([1, 65, 65 ** 2])
    inside_first = dens[vi] > iso       # the edge's first end is the dense one
    sign = np.where(inside_first, 1.0, -1.0)
    out_dir = np.zeros((codes.size, 3))
    out_dir[np.arange(codes.size), ax] = sign
    p = verts[tris]
    n = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    o = out_dir[tris].sum(1)
    return float(np.mean(np.einsum("ij,ij->i", n, o) > 0)), step


def test_mesh_matches_oracle_vertices_and_is_watertight():
    import torch  # noqa: F401

    oc, rc = paired_config(L=8, T=2 ** 12, growth=1.5)
    half = np.array([0.5, 0.4, 0.45], np.float32)
    rng = np.random.default_rng(3)
    p = O.init_params(oc, 4)
    nh = O.hash_param_count(oc)
    p[:nh] = rng.uniform(-2, 2, nh)
    p = p.astype(np.float32).astype(np.float64)
    ctx = Ctx(rc)
    try:
        oid = ctx.create(half=tuple(half), seed=4)
        ctx.set_state(oid, p)
        dens = _lattice(ctx, oid)
        ref = O.density_lattice(oc, p, half)
        assert np.max(np.abs(dens - ref) / ref) < 2e-5
        iso = float(np.median(dens))
        t0 = time.perf_counter()
        verts, tris = _extract(ctx, oid, iso)
        ms = (time.perf_counter() - t0) * 1e3
        codes, pos = O.mesh_vertices(dens.astype(np.float64), half, iso)
        print(f"\n{len(verts)} vertices, {len(tris)} triangles ({ms:.1f} ms including two host round trips)")
        assert len(verts) == codes.size and len(tris) > 1000
        assert np.max(np.abs(verts - pos)) < 2e-6
        assert tris.min() >= 0 and tris.max() < len(verts)
        _edge_check(codes, tris, dens, iso)
        # orientation from the lattice geometry (each vertex at its edge's midpoint, as the case table is built):
        # no triangle faces inwards (interpolated positions of a noisy field can twist a few slivers)
        vi, ax = codes // 3, codes % 3
        mid = np.stack([vi % 65, (vi // 65) % 65, vi // 65 ** 2], 1).astype(np.float64)
        mid[np.arange(codes.size), ax] += 0.5
        pm = mid[tris]
        n = np.cross(pm[:, 1] - pm[:, 0], pm[:, 2] - pm[:, 0])
        out = np.zeros((codes.size, 3))
        out[np.arange(codes.size), ax] = np.where(dens[vi] > iso, 1.0, -1.0)
        dots = np.einsum("ij,ij->i", n, out[tris].sum(1))
        assert np.all(dots >= -1e-9) and dots.sum() > 0
        frac, _ = _outward_fraction(verts.astype(np.float64), tris, codes, dens, iso)
        print(f"interpolated-geometry outward fraction {frac:.4f}")
        # too small buffers: the counts and CAPACITY, nothing written
        nv, nt = C.c_int64(), C.c_int64()
        v1 = np.zeros((4, 3), np.float32)
        t1 = np.full((4, 3), -7, np.int32)
        st = R.romap_extract_mesh(ctx.h, oid, iso, v1.ctypes.data, 4, t1.ctypes.data, 4, C.byref(nv), C.byref(nt), 0)
        assert st == R.ROMAP_ERR_CAPACITY and nv.value == len(verts) and nt.value == len(tris)
        assert np.all(t1 == -7)
        # device outputs
        import torch
        dv = torch.zeros((len(verts), 3), device="cuda")
        dt = torch.zeros((len(tris), 3), dtype=torch.int32, device="cuda")
        R.check(R.romap_extract_mesh(ctx.h, oid, iso, dv.data_ptr(), len(verts), dt.data_ptr(), len(tris), None, None,
                                     R.ROMAP_DEVICE_PTR))
        torch.cuda.synchronize()
        assert np.array_equal(dv.cpu().numpy(), verts) and np.array_equal(dt.cpu().numpy(), tris)
    finally:
        ctx.close()


def test_sphere_is_closed_with_euler_characteristic_two():
    """One dense level (N = 16) holding c - |v|^2 at its vertices, unit 0 = feature 0, output 0 = unit 0: sigma =
    exp(relu(interpolated c - |x|^2)); at iso exp(c - r^2) the surface is close to the sphere of radius r."""
    import torch  # noqa: F401

    oc, rc = paired_config(L=1, T=2 ** 13, n_min=16, growth=2.0)
    half = np.full(3, 0.5, np.float32)
    nh = O.hash_param_count(oc)
    p = np.zeros(O.param_count(oc))
    c, r = 0.2, 0.3
    for z in range(17):
        for y in range(17):
            for x in range(17):
                v = np.array([x, y, z]) / 16 - 0.5
                p[O.grid_index(oc, 0, x, y, z) * 2] = c - v @ v
    p[nh + O.mlp_layer_offset(oc, 0)] = 1.0
    p[nh + O.mlp_layer_offset(oc, 1)] = 1.0
    ctx = Ctx(rc)
    try:
        oid = ctx.create(seed=0)
        ctx.set_state(oid, p)
        iso = float(np.exp(c - r * r))
        verts, tris = _extract(ctx, oid, iso)
        dens = _lattice(ctx, oid)
        codes, _ = O.mesh_vertices(dens.astype(np.float64), half, iso)
        directed = _edge_check(codes, tris, dens, iso)
        assert all((w, u) in directed for (u, w) in directed)  # closed: no boundary edges
        E = len(directed) // 2
        chi = len(verts) - E + len(tris)
        rad = np.linalg.norm(verts, axis=1)
        print(f"\nsphere: V={len(verts)} E={E} F={len(tris)} chi={chi}; radius {rad.min():.4f}..{rad.max():.4f}")
        assert chi == 2
        assert np.all(np.abs(rad - r) < 0.01)
        frac, _ = _outward_fraction(verts.astype(np.float64), tris, codes, dens, iso)
        assert frac > 0.99
        # outward: the enclosed volume (divergence theorem) is positive and close to the ball's
        pv = verts[tris].astype(np.float64)
        vol = np.einsum("ij,ij->i", pv[:, 0], np.cross(pv[:, 1], pv[:, 2])).sum() / 6.0
        # (the vertices sit slightly inside radius r: trilinear interpolation of |x|^2 on the 16-grid overestimates
        # it, and linear interpolation of the exponential along lattice edges pulls towards the dense end)
        assert vol == pytest.approx(4.0 / 3.0 * np.pi * rad.mean() ** 3, rel=0.015)
    finally:
        ctx.close()
