// rgeo_scene_build.cpp -- host construction of the scene acceleration structures.
//
// * One BVH over every primitive of the scene, spheres and triangles, built
//   top-down with binned surface-area-heuristic splits (12 bins on the longest
//   centroid axis).  Children of a node are stored next to each other so a node
//   needs one child index.  Node boxes are padded by a few float32 ulps so that
//   the single-precision slab test on the device never rejects a box that the
//   segment touches.
// * A uniform grid of lower bounds on the Euclidean distance from any point of a
//   cell to the scene.  Cells overlapped by the bounding box of a primitive are
//   marked; the exact box-to-box distance from a cell to the nearest marked cell
//   equals the Euclidean distance to the nearest cell of the marked set dilated by
//   one cell per axis, which is computed with the separable squared distance
//   transform of Felzenszwalb and Huttenlocher ("Distance transforms of sampled
//   functions", 2012).  The tracer skips segment tests exactly while the polygon
//   stays inside a ball around its last query point whose radius is this bound
//   (Section 4.1 tests every segment; skipping provably empty ones changes no hit).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "rgeo_internal.h"

namespace rgeo {
namespace {

struct Box {
  float lo[3], hi[3];
  void reset() {
    for (int i = 0; i < 3; i++) {
      lo[i] = std::numeric_limits<float>::infinity();
      hi[i] = -std::numeric_limits<float>::infinity();
    }
  }
  void grow(const Box &b) {
    for (int i = 0; i < 3; i++) {
      lo[i] = std::min(lo[i], b.lo[i]);
      hi[i] = std::max(hi[i], b.hi[i]);
    }
  }
  void grow(const float p[3]) {
    for (int i = 0; i < 3; i++) {
      lo[i] = std::min(lo[i], p[i]);
      hi[i] = std::max(hi[i], p[i]);
    }
  }
  float area() const {
    float d[3];
    for (int i = 0; i < 3; i++) d[i] = std::max(0.0f, hi[i] - lo[i]);
    return 2.0f * (d[0] * d[1] + d[1] * d[2] + d[2] * d[0]);
  }
};

struct Prim {
  Box box;
  float c[3];
  int idx;
};

struct Builder {
  std::vector<Prim> prims;
  std::vector<Box> node_box;
  std::vector<int> node_first, node_count;  // count 0: internal, first = left child
  int max_depth = kMaxBvhDepth;
  int depth_seen = 0;

  int alloc_node() {
    node_box.emplace_back();
    node_first.push_back(0);
    node_count.push_back(0);
    return (int)node_box.size() - 1;
  }

  void build(int id, int first, int count, int depth) {
    depth_seen = std::max(depth_seen, depth);
    Box b, cb;
    b.reset();
    cb.reset();
    for (int i = first; i < first + count; i++) {
      b.grow(prims[i].box);
      cb.grow(prims[i].c);
    }
    node_box[id] = b;
    if (count <= 4 || depth >= max_depth) {
      node_first[id] = first;
      node_count[id] = count;
      return;
    }
    int axis = 0;
    float ext = cb.hi[0] - cb.lo[0];
    for (int i = 1; i < 3; i++)
      if (cb.hi[i] - cb.lo[i] > ext) {
        ext = cb.hi[i] - cb.lo[i];
        axis = i;
      }
    int mid;
    if (!(ext > 0.0f)) {
      mid = first + count / 2;  // all centroids coincide: split the list in half
    } else {
      constexpr int NB = 12;
      Box bb[NB];
      int bc[NB] = {0};
      for (auto &x : bb) x.reset();
      auto bin_of = [&](const Prim &p) {
        int k = (int)((p.c[axis] - cb.lo[axis]) / ext * NB);
        return std::min(std::max(k, 0), NB - 1);
      };
      for (int i = first; i < first + count; i++) {
        int k = bin_of(prims[i]);
        bb[k].grow(prims[i].box);
        bc[k]++;
      }
      float right_area[NB];
      int right_count[NB];
      Box acc;
      acc.reset();
      int n = 0;
      for (int k = NB - 1; k > 0; k--) {
        if (bc[k]) acc.grow(bb[k]);
        n += bc[k];
        right_area[k] = n ? acc.area() : 0.0f;
        right_count[k] = n;
      }
      acc.reset();
      n = 0;
      float best = std::numeric_limits<float>::infinity();
      int best_k = -1;
      for (int k = 1; k < NB; k++) {
        if (bc[k - 1]) acc.grow(bb[k - 1]);
        n += bc[k - 1];
        if (n == 0 || right_count[k] == 0) continue;
        float cost = acc.area() * n + right_area[k] * right_count[k];
        if (cost < best) {
          best = cost;
          best_k = k;
        }
      }
      if (best_k < 0) {
        mid = first + count / 2;
      } else {
        auto it = std::partition(prims.begin() + first, prims.begin() + first + count,
                                 [&](const Prim &p) { return bin_of(p) < best_k; });
        mid = (int)(it - prims.begin());
        if (mid == first || mid == first + count) mid = first + count / 2;
      }
    }
    int l = alloc_node();
    int r = alloc_node();
    (void)r;
    node_first[id] = l;
    node_count[id] = 0;
    build(l, first, mid - first, depth + 1);
    build(l + 1, mid, first + count - mid, depth + 1);
  }
};

inline float int_bits(int v) {
  float f;
  std::memcpy(&f, &v, 4);
  return f;
}

}  // namespace

bool build_bvh(const float *spheres, int n_spheres, const float *verts, int n_verts, const int32_t *tris,
               int n_tris, HostBVH &out, int max_depth) {
  out.nodes.clear();
  out.prims.clear();
  out.depth = 0;
  const int n = n_spheres + n_tris;
  if (n <= 0) return true;
  Builder B;
  B.max_depth = max_depth;
  B.prims.resize(n);
  for (int s = 0; s < n_spheres; s++) {
    Prim &p = B.prims[s];
    for (int i = 0; i < 3; i++) {
      p.box.lo[i] = spheres[4 * s + i] - spheres[4 * s + 3];
      p.box.hi[i] = spheres[4 * s + i] + spheres[4 * s + 3];
      p.c[i] = spheres[4 * s + i];
    }
    p.idx = s;  // object id: sphere index
  }
  for (int t = 0; t < n_tris; t++) {
    Prim &p = B.prims[n_spheres + t];
    p.box.reset();
    for (int v = 0; v < 3; v++) {
      int vi = tris[3 * t + v];
      if (vi < 0 || vi >= n_verts) return false;
      p.box.grow(verts + 3 * vi);
    }
    for (int i = 0; i < 3; i++) p.c[i] = 0.5f * (p.box.lo[i] + p.box.hi[i]);
    p.idx = n_spheres + t;  // object id: S + triangle index
  }
  int root = B.alloc_node();
  B.build(root, 0, n, 0);
  out.depth = B.depth_seen;
  const int nn = (int)B.node_box.size();
  out.nodes.resize(2 * nn);
  for (int k = 0; k < nn; k++) {
    const Box &b = B.node_box[k];
    float lo[3], hi[3];
    for (int i = 0; i < 3; i++) {
      float pad = 4e-6f * std::max(1.0f, std::max(std::fabs(b.lo[i]), std::fabs(b.hi[i])));
      lo[i] = b.lo[i] - pad;
      hi[i] = b.hi[i] + pad;
    }
    out.nodes[2 * k] = make_float4(lo[0], lo[1], lo[2], int_bits(B.node_first[k]));
    out.nodes[2 * k + 1] = make_float4(hi[0], hi[1], hi[2], int_bits(B.node_count[k]));
  }
  out.prims.resize(3 * n);
  for (int q = 0; q < n; q++) {
    const int id = B.prims[q].idx;
    if (id < n_spheres) {
      const float *sp = spheres + 4 * id;
      out.prims[3 * q] = make_float4(sp[0], sp[1], sp[2], int_bits(id));
      out.prims[3 * q + 1] = make_float4(sp[3], 0.0f, 0.0f, 0.0f);
      out.prims[3 * q + 2] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    } else {
      const int t = id - n_spheres;
      const float *a = verts + 3 * tris[3 * t];
      const float *b = verts + 3 * tris[3 * t + 1];
      const float *c = verts + 3 * tris[3 * t + 2];
      out.prims[3 * q] = make_float4(a[0], a[1], a[2], int_bits(id));
      out.prims[3 * q + 1] = make_float4(b[0], b[1], b[2], 0.0f);
      out.prims[3 * q + 2] = make_float4(c[0], c[1], c[2], 0.0f);
    }
  }
  return true;
}

namespace {

// Squared distance transform of a sampled function along one line
// (lower envelope of parabolas rooted at the samples).
void dt1d(const double *f, int n, double *d, std::vector<int> &v, std::vector<double> &z) {
  v.resize(n);
  z.resize(n + 1);
  int k = 0;
  v[0] = 0;
  z[0] = -std::numeric_limits<double>::infinity();
  z[1] = std::numeric_limits<double>::infinity();
  for (int q = 1; q < n; q++) {
    double s;
    for (;;) {
      int p = v[k];
      s = ((f[q] + (double)q * q) - (f[p] + (double)p * p)) / (2.0 * q - 2.0 * p);
      if (s <= z[k] && k > 0) {
        k--;
        continue;
      }
      break;
    }
    if (s <= z[k]) {  // k == 0 and the new parabola dominates everywhere
      v[0] = q;
      z[0] = -std::numeric_limits<double>::infinity();
      z[1] = std::numeric_limits<double>::infinity();
      continue;
    }
    k++;
    v[k] = q;
    z[k] = s;
    z[k + 1] = std::numeric_limits<double>::infinity();
  }
  k = 0;
  for (int q = 0; q < n; q++) {
    while (z[k + 1] < q) k++;
    double dq = (double)q - v[k];
    d[q] = dq * dq + f[v[k]];
  }
}

}  // namespace

void build_safe_grid(const float *spheres, int S, const float *verts, const int32_t *tris, int T,
                     int res, HostGrid &out) {
  out.dist.clear();
  out.dim[0] = out.dim[1] = out.dim[2] = 0;
  if (S + T == 0) return;
  Box sb;
  sb.reset();
  std::vector<Box> boxes;
  boxes.reserve(S + T);
  for (int s = 0; s < S; s++) {
    Box b;
    for (int i = 0; i < 3; i++) {
      b.lo[i] = spheres[4 * s + i] - spheres[4 * s + 3];
      b.hi[i] = spheres[4 * s + i] + spheres[4 * s + 3];
    }
    boxes.push_back(b);
    sb.grow(b);
  }
  for (int t = 0; t < T; t++) {
    Box b;
    b.reset();
    for (int v = 0; v < 3; v++) b.grow(verts + 3 * tris[3 * t + v]);
    boxes.push_back(b);
    sb.grow(b);
  }
  float ext = 0.0f;
  for (int i = 0; i < 3; i++) ext = std::max(ext, sb.hi[i] - sb.lo[i]);
  float cell = std::max(ext, 1e-3f) / (float)res;
  for (int i = 0; i < 3; i++) {
    out.smin[i] = sb.lo[i];
    out.smax[i] = sb.hi[i];
    out.gmin[i] = sb.lo[i] - cell;
    out.dim[i] = (int)std::ceil((sb.hi[i] - sb.lo[i]) / cell) + 3;
  }
  out.cell = cell;
  const int nx = out.dim[0], ny = out.dim[1], nz = out.dim[2];
  const size_t N = (size_t)nx * ny * nz;
  std::vector<unsigned char> mark(N, 0);
  auto clampi = [](int v, int lo, int hi) { return std::min(std::max(v, lo), hi); };
  for (const Box &b : boxes) {
    int lo[3], hi[3];
    for (int i = 0; i < 3; i++) {
      // dilate by one cell per axis while marking (see the header comment)
      lo[i] = clampi((int)std::floor((b.lo[i] - out.gmin[i]) / cell) - 1, 0, out.dim[i] - 1);
      hi[i] = clampi((int)std::floor((b.hi[i] - out.gmin[i]) / cell) + 1, 0, out.dim[i] - 1);
    }
    for (int z = lo[2]; z <= hi[2]; z++)
      for (int y = lo[1]; y <= hi[1]; y++)
        for (int x = lo[0]; x <= hi[0]; x++) mark[((size_t)z * ny + y) * nx + x] = 1;
  }
  const double BIG = 1e20;
  std::vector<double> f(N);
  for (size_t i = 0; i < N; i++) f[i] = mark[i] ? 0.0 : BIG;
  int nmax = std::max(nx, std::max(ny, nz));
  std::vector<double> line(nmax), res1(nmax);
  std::vector<int> v;
  std::vector<double> zz;
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++) {
      double *row = &f[((size_t)z * ny + y) * nx];
      for (int x = 0; x < nx; x++) line[x] = row[x];
      dt1d(line.data(), nx, res1.data(), v, zz);
      for (int x = 0; x < nx; x++) row[x] = res1[x];
    }
  for (int z = 0; z < nz; z++)
    for (int x = 0; x < nx; x++) {
      for (int y = 0; y < ny; y++) line[y] = f[((size_t)z * ny + y) * nx + x];
      dt1d(line.data(), ny, res1.data(), v, zz);
      for (int y = 0; y < ny; y++) f[((size_t)z * ny + y) * nx + x] = res1[y];
    }
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      for (int z = 0; z < nz; z++) line[z] = f[((size_t)z * ny + y) * nx + x];
      dt1d(line.data(), nz, res1.data(), v, zz);
      for (int z = 0; z < nz; z++) f[((size_t)z * ny + y) * nx + x] = res1[z];
    }
  out.dist.resize(N);
  for (size_t i = 0; i < N; i++) {
    double d = std::sqrt(std::min(f[i], BIG)) * cell;
    // margin for float32 rounding of the tracer's accumulated segment lengths
    double lb = d * (1.0 - 1e-5) - 1e-4;
    out.dist[i] = (float)std::max(0.0, lb);
  }
}

}  // namespace rgeo
