"""The marching-cubes case table of the library, checked by brute force on every case: triangles use exactly the
crossed edges, each case's triangles form a surface whose open boundary lies on the cube's faces, every triangle
faces from the inside corners to the outside ones, and two cubes that share a face cut it with the same segments
whatever their other corners (no cracks between cubes)."""
import itertools

import numpy as np
import pytest

from paper_2304_05735_gb300 import romap as R

ROW = 16


def edge_corners(e):
    d, q = divmod(e, 4)
    o = sorted([(d + 1) % 3, (d + 2) % 3])
    base = ((q & 1) << o[0]) | (((q >> 1) & 1) << o[1])
    return base, base | (1 << d)


def pos(c):
    return np.array([(c >> a) & 1 for a in range(3)], np.float64)


def faces_of_edge(e):
    """The two faces (axis, side) that contain edge e."""
    a, _ = edge_corners(e)
    d = e // 4
    return {(ax, (a >> ax) & 1) for ax in range(3) if ax != d}


@pytest.fixture(scope="module")
def table():
    t = np.zeros((256, ROW), np.int8)
    c = np.zeros(256, np.uint8)
    assert R.romap_mc_case_table(t.ctypes.data, c.ctypes.data) == R.ROMAP_OK
    return t, c


def tris_of(t, c, cs):
    return [tuple(int(x) for x in t[cs, 3 * i:3 * i + 3]) for i in range(int(c[cs]))]


def test_crossed_edges_and_terminator(table):
    t, c = table
    for cs in range(256):
        inside = [(cs >> k) & 1 for k in range(8)]
        crossed = {e for e in range(12) if inside[edge_corners(e)[0]] != inside[edge_corners(e)[1]]}
        used = {e for tri in tris_of(t, c, cs) for e in tri}
        assert used == crossed, cs
        assert t[cs, 3 * c[cs]] == -1 or 3 * c[cs] == ROW - 1
    assert c[0] == 0 and c[255] == 0 and c.max() <= 5


def test_case_surfaces_close_on_the_cube_faces_and_face_outwards(table):
    t, c = table
    for cs in range(256):
        inside = [(cs >> k) & 1 for k in range(8)]
        count = {}
        total = 0.0
        for tri in tris_of(t, c, cs):
            for i in range(3):
                a, b = tri[i], tri[(i + 1) % 3]
                count[(a, b)] = count.get((a, b), 0) + 1
            # orientation: the normal of the midpoint triangle points from inside to outside corners
            m = [0.5 * (pos(edge_corners(e)[0]) + pos(edge_corners(e)[1])) for e in tri]
            n = np.cross(m[1] - m[0], m[2] - m[0])
            out = sum((pos(edge_corners(e)[1]) - pos(edge_corners(e)[0])) * (1 if inside[edge_corners(e)[0]] else -1)
                      for e in tri)
            assert n @ out >= -1e-12, (cs, tri)  # never inward (a fan triangle of a skew loop may be edge-on)
            total += n @ out
        assert c[cs] == 0 or total > 0, cs
        for (a, b), k in count.items():
            if (b, a) in count:
                assert k == 1 and count[(b, a)] == 1, (cs, a, b)  # interior edge: once each way
            else:
                assert k == 1 and faces_of_edge(a) & faces_of_edge(b), (cs, a, b)  # boundary edge on a face


def face_segments(t, c, cs, face):
    """Boundary segments of case cs lying on face (axis, side), as unordered pairs of the face's edges."""
    segs = set()
    count = {}
    for tri in tris_of(t, c, cs):
        for i in range(3):
            count[(tri[i], tri[(i + 1) % 3])] = 1
    for (a, b) in count:
        if (b, a) not in count and face in (faces_of_edge(a) & faces_of_edge(b)):
            segs.add(frozenset((a, b)))
    return segs


def test_shared_faces_are_cut_alike(table):
    """Cube A's +x face is cube B's -x face: with the same 4 corners there, both draw the same segments."""
    t, c = table
    rng = np.random.default_rng(0)
    # corners of the +x face of A (bit 0 = 1) correspond to B's corners with bit 0 = 0
    for face_bits in range(16):
        for _ in range(8):
            a_rest, b_rest = rng.integers(0, 2, 4), rng.integers(0, 2, 4)
            a_case = b_case = 0
            for k, (y, z) in enumerate(itertools.product((0, 1), (0, 1))):
                f = (face_bits >> k) & 1
                ca_face, ca_other = 1 | (y << 1) | (z << 2), 0 | (y << 1) | (z << 2)
                cb_face, cb_other = 0 | (y << 1) | (z << 2), 1 | (y << 1) | (z << 2)
                a_case |= (f << ca_face) | (int(a_rest[k]) << ca_other)
                b_case |= (f << cb_face) | (int(b_rest[k]) << cb_other)
            # map A's +x-face edges (x = 1) to B's -x-face edges (x = 0): same y/z edge, other side in x
            to_b = {}
            for e in range(12):
                a0, a1 = edge_corners(e)
                if (a0 & 1) and (a1 & 1):
                    for e2 in range(12):
                        b0, b1 = edge_corners(e2)
                        if {b0, b1} == {a0 & ~1, a1 & ~1}:
                            to_b[e] = e2
            sa = {frozenset(to_b[x] for x in seg) for seg in face_segments(t, c, a_case, (0, 1))}
            sb = face_segments(t, c, b_case, (0, 0))
            assert sa == sb, (face_bits, a_case, b_case)
