// Marching-cubes case table (Lorensen & Cline 1987), built at load time by construction rather than typed in.
//
// Cube corners c = 0..7 sit at (c & 1, (c >> 1) & 1, (c >> 2) & 1).  Edge e = 4 d + q runs along axis d from the
// corner with bit d = 0 to the one with bit d = 1; q enumerates the other two axes' bits (lower axis first).  A corner
// is "inside" when its density exceeds the iso-level.  For each of the 256 inside/outside patterns:
//   1. on each of the 6 faces, the edges whose end corners differ are joined in pairs by segments: with 2 such edges,
//      to each other; with 4 (diagonal corners alike) each inside corner is cut off by the segment joining its two
//      edges on that face.  The rule depends only on the face's 4 corners, so the two cubes sharing a face draw the
//      same segments and the mesh has no cracks;
//   2. every crossed edge lies on two faces, so the segments close into loops; each loop is oriented so that its
//      normal (Newell's formula over the edge midpoints) points from the inside corners of its edges to the outside
//      ones, and is split into a fan of triangles.
// The table lists per case up to kMcMaxTri triangles as edge triples, -1 terminated.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <vector>

#include "romap.h"
#include "romap_internal.cuh"

namespace romap {

namespace {

struct Edge {
  int a, b;  // end corners (bit d of a is 0, of b is 1)
};

Edge edge_corners(int e) {
  const int d = e / 4, q = e % 4;
  const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
  const int lo = o1 < o2 ? o1 : o2, hi = o1 < o2 ? o2 : o1;
  const int base = ((q & 1) << lo) | (((q >> 1) & 1) << hi);
  return Edge{base, base | (1 << d)};
}

int edge_of(int c0, int c1) {
  for (int e = 0; e < 12; ++e) {
    const Edge E = edge_corners(e);
    if ((E.a == c0 && E.b == c1) || (E.a == c1 && E.b == c0)) return e;
  }
  return -1;
}

void corner_pos(int c, double p[3]) {
  for (int a = 0; a < 3; ++a) p[a] = (double)((c >> a) & 1);
}

}  // namespace

int build_mc_table(int8_t table[256][3 * kMcMaxTri + 1], uint8_t counts[256]) {
  int worst = 0;
  for (int cs = 0; cs < 256; ++cs) {
    auto inside = [&](int c) { return ((cs >> c) & 1) != 0; };
    // segments on the faces
    std::vector<int> nb[12];
    for (int d = 0; d < 3; ++d)
      for (int side = 0; side < 2; ++side) {
        const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
        // face corners in cyclic order
        int cyc[4];
        const int fix = side << d;
        cyc[0] = fix;
        cyc[1] = fix | (1 << o1);
        cyc[2] = fix | (1 << o1) | (1 << o2);
        cyc[3] = fix | (1 << o2);
        int fe[4];
        bool cross[4];
        int n_cross = 0;
        for (int k = 0; k < 4; ++k) {
          fe[k] = edge_of(cyc[k], cyc[(k + 1) % 4]);  // edge between corner k and k+1
          cross[k] = inside(cyc[k]) != inside(cyc[(k + 1) % 4]);
          n_cross += cross[k] ? 1 : 0;
        }
        auto join = [&](int e0, int e1) {
          nb[e0].push_back(e1);
          nb[e1].push_back(e0);
        };
        if (n_cross == 2) {
          int f[2], m = 0;
          for (int k = 0; k < 4; ++k)
            if (cross[k]) f[m++] = fe[k];
          join(f[0], f[1]);
        } else if (n_cross == 4) {
          for (int k = 0; k < 4; ++k)
            if (inside(cyc[k])) join(fe[(k + 3) % 4], fe[k]);  // the two face edges at inside corner k
        }
      }
    // loops
    bool used[12] = {false};
    std::vector<int8_t> tris;
    for (int start = 0; start < 12; ++start) {
      if (used[start] || nb[start].empty()) continue;
      if (nb[start].size() != 2) return -1;  // every crossed edge lies on exactly two faces
      std::vector<int> loop;
      int prev = -1, cur = start;
      while (true) {
        loop.push_back(cur);
        used[cur] = true;
        const int next = nb[cur][0] != prev ? nb[cur][0] : nb[cur][1];
        prev = cur;
        cur = next;
        if (cur == start) break;
        if (used[cur] || loop.size() > 12) return -1;
      }
      // orientation: Newell normal of the midpoint polygon against (outside - inside) of the loop's edges
      double nrm[3] = {0, 0, 0}, dir[3] = {0, 0, 0};
      const size_t n = loop.size();
      std::vector<std::array<double, 3>> mid(n);
      for (size_t i = 0; i < n; ++i) {
        const Edge E = edge_corners(loop[i]);
        double pa[3], pb[3];
        corner_pos(E.a, pa);
        corner_pos(E.b, pb);
        const bool a_in = inside(E.a);
        for (int a = 0; a < 3; ++a) {
          mid[i][a] = 0.5 * (pa[a] + pb[a]);
          dir[a] += a_in ? (pb[a] - pa[a]) : (pa[a] - pb[a]);
        }
      }
      for (size_t i = 0; i < n; ++i) {
        const auto& p = mid[i];
        const auto& q = mid[(i + 1) % n];
        nrm[0] += (p[1] - q[1]) * (p[2] + q[2]);
        nrm[1] += (p[2] - q[2]) * (p[0] + q[0]);
        nrm[2] += (p[0] - q[0]) * (p[1] + q[1]);
      }
      if (nrm[0] * dir[0] + nrm[1] * dir[1] + nrm[2] * dir[2] < 0.0) std::reverse(loop.begin(), loop.end());
      for (size_t i = 1; i + 1 < n; ++i) {
        tris.push_back((int8_t)loop[0]);
        tris.push_back((int8_t)loop[i]);
        tris.push_back((int8_t)loop[i + 1]);
      }
    }
    const int nt = (int)tris.size() / 3;
    if (nt > kMcMaxTri) return -1;
    worst = nt > worst ? nt : worst;
    counts[cs] = (uint8_t)nt;
    for (int i = 0; i < 3 * kMcMaxTri + 1; ++i) table[cs][i] = i < (int)tris.size() ? tris[i] : (int8_t)-1;
  }
  return worst;
}

}  // namespace romap

extern "C" ROMAP_API romap_status romap_mc_case_table(int8_t* triangles, uint8_t* counts) {
  if (!triangles || !counts) return ROMAP_ERR_INVALID_ARG;
  static int8_t t[256][3 * romap::kMcMaxTri + 1];
  static uint8_t c[256];
  if (romap::build_mc_table(t, c) < 0) return ROMAP_ERR_BAD_STATE;
  for (int cs = 0; cs < 256; ++cs) {
    counts[cs] = c[cs];
    for (int i = 0; i < 3 * romap::kMcMaxTri + 1; ++i) triangles[cs * (3 * romap::kMcMaxTri + 1) + i] = t[cs][i];
  }
  return ROMAP_OK;
}
