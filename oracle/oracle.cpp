// CPU checker for the improved-BVH ray tracer (arxiv 2208.10008).
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg load this library.  The CUDA path never calls
// it, links it or includes anything from here, and this file includes
// nothing from the CUDA path.
//
// Everything is plain, slow and in float64.  Float32 inputs (triangle
// vertices, rays) are promoted exactly to float64 before any arithmetic.
// Build with -ffp-contract=off: the triangle test below fixes its operation
// order and must not be fused into FMAs.
//
// Contents
//  1. tri_hit        Moller-Trumbore ray/triangle test (the hit rule).
//  2. brute force    every ray against every triangle: the plain definition
//                    of the closest hit the method must reproduce (Sec. I;
//                    Sec. IV.B: accelerated paths equal unaccelerated ones).
//  3. BVH build      top-down recursive build of Sec. II.C (Fig. 2) with the
//                    hybrid SAH + distance split cost of Eq. 2 (Eq. 1 at
//                    alpha = 1), AABBs of Eq. 3, exact sweep over all object
//                    splits on the three axes, leaf when count <= max_leaf.
//  4. BVH walk       collision detection of Sec. III.B (Fig. 4): box test,
//                    descend, test leaf triangles, keep the nearest hit.
//  5. tree cost      Eq. 2 applied recursively to score any binary tree.
//  6. reflection     specular bounce of Sec. III.B.
//  7. launch dirs    icosahedral subdivision of Sec. III.A; Fibonacci sphere.
//  8. reception      receiving sphere of Sec. III.C (Eq. 4), every path
//                    segment against every receiver.
//
// Readings of points the paper leaves open (all documented with the design):
//  * hit rule: edges inclusive (u >= 0, v >= 0, u + v <= 1); |det| <=
//    1e-14 |e1||e2||d| counts as parallel (miss); valid iff tmin < t < tmax;
//    equal t -> lowest triangle id wins; rays with a non-finite component or
//    tmax <= tmin miss.
//  * Eq. 2 distance: d^2 = (d_A^2 + d_B^2) / 2 with d_X the distance from the
//    centre of AABB X to the source point; optional normalisation
//    (dist_norm = 1) d^2 / diag(C)^2 * k_C * t_i, or the count-weighted
//    scale-free form (dist_norm = 2) (k_A d_A^2 + k_B d_B^2) / diag(C)^2 * t_i,
//    which weights each child's distance by its triangles as the SAH term
//    weights its area.
//  * Eq. 3 boxes are closed (min <= x <= max).
//  * Eq. 4 reception: a segment t in [tmin, tend) of ray (o, d) (tend = the
//    nearer of its hit and tmax) receives at point p when the foot of the
//    perpendicular from p, t* = (p - o).d / (d.d), lies in [tmin, tend) and
//    |p - (o + t* d)| <= l delta / sqrt(3) with l = (range0 - tmax) + t*:
//    the path length from the source, since every bounce leaves the
//    remaining range in tmax (directions have unit length).
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

const double kInf = std::numeric_limits<double>::infinity();

struct V3 {
  double x, y, z;
};

inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
// Fixed evaluation order: (a.x*b.x + a.y*b.y) + a.z*b.z.
inline double dot(V3 a, V3 b) {
  double s = a.x * b.x;
  s = s + a.y * b.y;
  s = s + a.z * b.z;
  return s;
}
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

inline V3 vert(const float* tris, int64_t i, int k) {
  const float* p = tris + i * 9 + k * 3;
  return {(double)p[0], (double)p[1], (double)p[2]};
}

struct Ray {
  V3 o, d;
  double tmin, tmax;
  bool valid;
};

inline Ray load_ray(const float* rays, int64_t r) {
  const float* p = rays + r * 8;
  Ray ray;
  ray.o = {(double)p[0], (double)p[1], (double)p[2]};
  ray.tmin = p[3];
  ray.d = {(double)p[4], (double)p[5], (double)p[6]};
  ray.tmax = p[7];
  bool fin = std::isfinite(ray.o.x) && std::isfinite(ray.o.y) && std::isfinite(ray.o.z) &&
             std::isfinite(ray.d.x) && std::isfinite(ray.d.y) && std::isfinite(ray.d.z) &&
             !std::isnan(ray.tmin) && !std::isnan(ray.tmax);
  ray.valid = fin && ray.tmax > ray.tmin;
  return ray;
}

// 1. Moller-Trumbore (Moller & Trumbore, JGT 1997), two-sided, inclusive
// edges.  Returns true when the ray's line meets the triangle; the caller
// applies the t interval.
bool tri_hit(const Ray& r, V3 v0, V3 v1, V3 v2, double* t, double* u, double* v) {
  V3 e1 = sub(v1, v0);
  V3 e2 = sub(v2, v0);
  V3 p = cross(r.d, e2);
  double det = dot(e1, p);
  double n1 = std::sqrt(dot(e1, e1));
  double n2 = std::sqrt(dot(e2, e2));
  double nd = std::sqrt(dot(r.d, r.d));
  double lim = 1e-14 * ((n1 * n2) * nd);
  if (std::fabs(det) <= lim) return false;
  double inv = 1.0 / det;
  V3 s = sub(r.o, v0);
  double uu = dot(s, p) * inv;
  if (uu < 0.0 || uu > 1.0) return false;
  V3 q = cross(s, e1);
  double vv = dot(r.d, q) * inv;
  if (vv < 0.0 || uu + vv > 1.0) return false;
  *t = dot(e2, q) * inv;
  *u = uu;
  *v = vv;
  return true;
}

struct Best {
  double t = kInf, t2 = kInf, u = 0, v = 0;
  int32_t id = -1;
  // Candidates arrive in any order; (t, id) lexicographic minimum wins.
  void offer(double tt, int32_t i, double uu, double vv) {
    if (tt < t || (tt == t && i < id)) {
      if (id >= 0) t2 = std::min(t2, t);
      t = tt;
      id = i;
      u = uu;
      v = vv;
    } else {
      t2 = std::min(t2, tt);
    }
  }
};

template <class F>
void parallel_for(int64_t n, int n_threads, F f) {
  if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (n <= 0) return;
  const int64_t chunk = 64;
  std::atomic<int64_t> next(0);
  auto work = [&]() {
    for (;;) {
      int64_t b = next.fetch_add(chunk);
      if (b >= n) break;
      int64_t e = std::min(n, b + chunk);
      for (int64_t i = b; i < e; ++i) f(i);
    }
  };
  if (n_threads == 1) {
    work();
    return;
  }
  std::vector<std::thread> th;
  for (int k = 0; k < n_threads; ++k) th.emplace_back(work);
  for (auto& x : th) x.join();
}

// ---------------------------------------------------------------- boxes
struct Box {
  double lo[3] = {kInf, kInf, kInf};
  double hi[3] = {-kInf, -kInf, -kInf};
  void add(V3 p) {
    double c[3] = {p.x, p.y, p.z};
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], c[a]);
      hi[a] = std::max(hi[a], c[a]);
    }
  }
  void add(const Box& b) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], b.lo[a]);
      hi[a] = std::max(hi[a], b.hi[a]);
    }
  }
  double area() const {
    double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
  }
};

Box tri_box(const float* tris, int64_t i) {
  Box b;
  for (int k = 0; k < 3; ++k) b.add(vert(tris, i, k));
  return b;
}

struct CostParams {
  double alpha, t_i, t_trav, src[3];
  int dist_norm;
};

// Eq. 2 (Eq. 1 when alpha = 1) for children A, B of parent C.
double eq2(const Box& A, double kA, const Box& B, double kB, const Box& C, const CostParams& p) {
  double sc = C.area();
  double sah;
  if (sc > 0.0)
    sah = (A.area() / sc) * kA * p.t_i + (B.area() / sc) * kB * p.t_i;
  else
    sah = (kA + kB) * p.t_i;
  double dA2 = 0.0, dB2 = 0.0, diag2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    double ca = 0.5 * (A.lo[a] + A.hi[a]) - p.src[a];
    double cb = 0.5 * (B.lo[a] + B.hi[a]) - p.src[a];
    double dc = C.hi[a] - C.lo[a];
    dA2 += ca * ca;
    dB2 += cb * cb;
    diag2 += dc * dc;
  }
  double d2 = 0.5 * (dA2 + dB2);
  if (p.dist_norm == 2)
    d2 = (diag2 > 0.0 ? (kA * dA2 + kB * dB2) / diag2 : 0.0) * p.t_i;
  else if (p.dist_norm)
    d2 = (diag2 > 0.0 ? d2 / diag2 : 0.0) * (kA + kB) * p.t_i;
  return p.alpha * sah + (1.0 - p.alpha) * d2 + p.t_trav;
}

// ---------------------------------------------------------------- BVH
struct Node {
  Box box;
  int32_t child[2] = {-1, -1};  // internal node indices; -1 for a leaf
  int64_t first = 0, count = 0; // leaf range in `prims`
};

struct Bvh {
  const float* tris = nullptr;  // caller keeps the triangles alive
  int64_t n_tri = 0;
  std::vector<Node> nodes;      // node 0 is the root
  std::vector<int32_t> prims;   // triangle ids in leaf order
  CostParams cp{};
  int max_leaf = 1;
  int depth = 0;
};

void build_bvh(Bvh& B) {
  const int64_t n = B.n_tri;
  std::vector<V3> cen(n);
  std::vector<Box> tb(n);
  for (int64_t i = 0; i < n; ++i) {
    V3 a = vert(B.tris, i, 0), b = vert(B.tris, i, 1), c = vert(B.tris, i, 2);
    cen[i] = {((a.x + b.x) + c.x) / 3.0, ((a.y + b.y) + c.y) / 3.0, ((a.z + b.z) + c.z) / 3.0};
    tb[i] = tri_box(B.tris, i);
  }
  B.prims.resize(n);
  for (int64_t i = 0; i < n; ++i) B.prims[i] = (int32_t)i;
  B.nodes.clear();
  B.nodes.emplace_back();
  struct Task {
    int32_t node;
    int64_t b, e;
    int depth;
  };
  std::vector<Task> stack{{0, 0, n, 1}};
  std::vector<Box> pre, suf;
  auto axis_key = [&](int ax, int32_t i) {
    return ax == 0 ? cen[i].x : (ax == 1 ? cen[i].y : cen[i].z);
  };
  while (!stack.empty()) {
    Task tk = stack.back();
    stack.pop_back();
    B.depth = std::max(B.depth, tk.depth);
    Box C;
    for (int64_t k = tk.b; k < tk.e; ++k) C.add(tb[B.prims[k]]);
    B.nodes[tk.node].box = C;
    const int64_t cnt = tk.e - tk.b;
    if (cnt <= B.max_leaf) {
      B.nodes[tk.node].first = tk.b;
      B.nodes[tk.node].count = cnt;
      continue;
    }
    double best = kInf;
    int best_ax = -1;
    int64_t best_i = -1;
    for (int ax = 0; ax < 3; ++ax) {
      std::sort(B.prims.begin() + tk.b, B.prims.begin() + tk.e, [&](int32_t x, int32_t y) {
        double kx = axis_key(ax, x), ky = axis_key(ax, y);
        return kx < ky || (kx == ky && x < y);
      });
      pre.assign(cnt + 1, Box());
      suf.assign(cnt + 1, Box());
      for (int64_t i = 0; i < cnt; ++i) {
        pre[i + 1] = pre[i];
        pre[i + 1].add(tb[B.prims[tk.b + i]]);
      }
      for (int64_t i = cnt - 1; i >= 0; --i) {
        suf[i] = suf[i + 1];
        suf[i].add(tb[B.prims[tk.b + i]]);
      }
      for (int64_t i = 1; i < cnt; ++i) {
        double c = eq2(pre[i], (double)i, suf[i], (double)(cnt - i), C, B.cp);
        if (c < best) {
          best = c;
          best_ax = ax;
          best_i = i;
        }
      }
    }
    if (best_ax < 0) {  // every cost NaN (non-finite input); split at the middle
      best_ax = 0;
      best_i = cnt / 2;
    }
    std::sort(B.prims.begin() + tk.b, B.prims.begin() + tk.e, [&](int32_t x, int32_t y) {
      double kx = axis_key(best_ax, x), ky = axis_key(best_ax, y);
      return kx < ky || (kx == ky && x < y);
    });
    int32_t l = (int32_t)B.nodes.size();
    B.nodes.emplace_back();
    int32_t r = (int32_t)B.nodes.size();
    B.nodes.emplace_back();
    B.nodes[tk.node].child[0] = l;
    B.nodes[tk.node].child[1] = r;
    stack.push_back({r, tk.b + best_i, tk.e, tk.depth + 1});
    stack.push_back({l, tk.b, tk.b + best_i, tk.depth + 1});
  }
}

// Slab test in float64 with the box and the interval widened by a tiny
// relative margin, so that a triangle the exact test hits is never skipped
// because of rounding in either computation.
bool slab(const Ray& r, const Box& b, double tlo, double thi, double* tnear) {
  const double o[3] = {r.o.x, r.o.y, r.o.z};
  const double d[3] = {r.d.x, r.d.y, r.d.z};
  double t0 = -kInf, t1 = kInf;
  for (int a = 0; a < 3; ++a) {
    double pad = 1e-9 * (std::fabs(b.lo[a]) + std::fabs(b.hi[a]) + std::fabs(o[a])) + 1e-12;
    double lo = b.lo[a] - pad, hi = b.hi[a] + pad;
    if (d[a] == 0.0) {
      if (o[a] < lo || o[a] > hi) return false;
      continue;
    }
    double ta = (lo - o[a]) / d[a];
    double tb = (hi - o[a]) / d[a];
    if (ta > tb) std::swap(ta, tb);
    t0 = std::max(t0, ta);
    t1 = std::min(t1, tb);
  }
  double slack0 = 1e-9 * std::fabs(t0), slack1 = 1e-9 * std::fabs(t1);
  if (t0 - slack0 > t1 + slack1) return false;
  if (t1 + slack1 < tlo) return false;
  if (t0 - slack0 > thi) return false;
  *tnear = t0;
  return true;
}

inline double widen(double t) { return t + 1e-9 * std::fabs(t); }

// 4. nearest hit (and second-nearest distance) through the BVH.
void walk_closest(const Bvh& B, const Ray& r, int32_t skip, Best* out) {
  Best best;
  if (!r.valid || B.nodes.empty()) {
    *out = best;
    return;
  }
  std::vector<int32_t> st;
  st.reserve(64);
  double tn;
  if (slab(r, B.nodes[0].box, r.tmin, widen(r.tmax), &tn)) st.push_back(0);
  while (!st.empty()) {
    int32_t ni = st.back();
    st.pop_back();
    const Node& nd = B.nodes[ni];
    double bound = widen(std::min(best.t2, r.tmax));
    if (nd.child[0] < 0) {
      for (int64_t k = nd.first; k < nd.first + nd.count; ++k) {
        int32_t id = B.prims[k];
        if (id == skip) continue;
        double t, u, v;
        if (tri_hit(r, vert(B.tris, id, 0), vert(B.tris, id, 1), vert(B.tris, id, 2), &t, &u, &v) &&
            t > r.tmin && t < r.tmax)
          best.offer(t, id, u, v);
      }
      continue;
    }
    double ta, tb;
    bool ha = slab(r, B.nodes[nd.child[0]].box, r.tmin, bound, &ta);
    bool hb = slab(r, B.nodes[nd.child[1]].box, r.tmin, bound, &tb);
    if (ha && hb) {
      if (ta <= tb) {
        st.push_back(nd.child[1]);
        st.push_back(nd.child[0]);
      } else {
        st.push_back(nd.child[0]);
        st.push_back(nd.child[1]);
      }
    } else if (ha) {
      st.push_back(nd.child[0]);
    } else if (hb) {
      st.push_back(nd.child[1]);
    }
  }
  *out = best;
}

bool walk_any(const Bvh& B, const Ray& r, int32_t skip) {
  if (!r.valid || B.nodes.empty()) return false;
  std::vector<int32_t> st;
  double tn;
  if (slab(r, B.nodes[0].box, r.tmin, widen(r.tmax), &tn)) st.push_back(0);
  while (!st.empty()) {
    const Node& nd = B.nodes[st.back()];
    st.pop_back();
    if (nd.child[0] < 0) {
      for (int64_t k = nd.first; k < nd.first + nd.count; ++k) {
        int32_t id = B.prims[k];
        if (id == skip) continue;
        double t, u, v;
        if (tri_hit(r, vert(B.tris, id, 0), vert(B.tris, id, 1), vert(B.tris, id, 2), &t, &u, &v) &&
            t > r.tmin && t < r.tmax)
          return true;
      }
      continue;
    }
    for (int s = 0; s < 2; ++s)
      if (slab(r, B.nodes[nd.child[s]].box, r.tmin, widen(r.tmax), &tn)) st.push_back(nd.child[s]);
  }
  return false;
}

}  // namespace

extern "C" {

int orc_version(void) { return 1; }

// Single triangle test: tri9 = 3 float32 vertices, ray8 = (o, tmin, d, tmax)
// as float32.  Returns 1 and (t, u, v) when the line meets the triangle under
// the hit rule, ignoring the t interval; 0 otherwise.
int orc_tri_hit(const float* tri9, const float* ray8, double* t, double* u, double* v) {
  Ray r = load_ray(ray8, 0);
  return tri_hit(r, vert(tri9, 0, 0), vert(tri9, 0, 1), vert(tri9, 0, 2), t, u, v) ? 1 : 0;
}

// 2. Brute force closest hit.  skip (nullable): per-ray triangle id to ignore.
// t2_out (nullable): distance of the second-nearest hit (another triangle).
int orc_closest_brute(const float* tris, int64_t n_tri, const float* rays, int64_t n_ray,
                      const int32_t* skip, double* t_out, int32_t* id_out, double* u_out,
                      double* v_out, double* t2_out, int n_threads) {
  parallel_for(n_ray, n_threads, [&](int64_t ri) {
    Ray r = load_ray(rays, ri);
    Best best;
    int32_t sk = skip ? skip[ri] : -1;
    if (r.valid) {
      for (int64_t i = 0; i < n_tri; ++i) {
        if (i == sk) continue;
        double t, u, v;
        if (tri_hit(r, vert(tris, i, 0), vert(tris, i, 1), vert(tris, i, 2), &t, &u, &v) &&
            t > r.tmin && t < r.tmax)
          best.offer(t, (int32_t)i, u, v);
      }
    }
    t_out[ri] = best.t;
    id_out[ri] = best.id;
    if (u_out) u_out[ri] = best.u;
    if (v_out) v_out[ri] = best.v;
    if (t2_out) t2_out[ri] = best.t2;
  });
  return 0;
}

int orc_any_brute(const float* tris, int64_t n_tri, const float* rays, int64_t n_ray,
                  const int32_t* skip, uint8_t* out, int n_threads) {
  parallel_for(n_ray, n_threads, [&](int64_t ri) {
    Ray r = load_ray(rays, ri);
    int32_t sk = skip ? skip[ri] : -1;
    uint8_t hit = 0;
    if (r.valid) {
      for (int64_t i = 0; i < n_tri && !hit; ++i) {
        if (i == sk) continue;
        double t, u, v;
        if (tri_hit(r, vert(tris, i, 0), vert(tris, i, 1), vert(tris, i, 2), &t, &u, &v) &&
            t > r.tmin && t < r.tmax)
          hit = 1;
      }
    }
    out[ri] = hit;
  });
  return 0;
}

// 3. Build.  The triangles must stay alive while the handle is used.
void* orc_bvh_build(const float* tris, int64_t n_tri, double alpha, double t_i, double t_trav,
                    const double* source3, int max_leaf, int dist_norm) {
  Bvh* B = new Bvh();
  B->tris = tris;
  B->n_tri = n_tri;
  B->cp = {alpha, t_i, t_trav, {source3[0], source3[1], source3[2]}, dist_norm};
  B->max_leaf = max_leaf < 1 ? 1 : max_leaf;
  if (n_tri > 0) build_bvh(*B);
  return B;
}

void orc_bvh_free(void* h) { delete static_cast<Bvh*>(h); }

// info[0..5] = nodes, leaves, depth, largest leaf, smallest leaf, prims.
int orc_bvh_info(void* h, int64_t* info) {
  const Bvh& B = *static_cast<Bvh*>(h);
  int64_t leaves = 0, big = 0, small = B.n_tri;
  for (const Node& n : B.nodes)
    if (n.child[0] < 0) {
      ++leaves;
      big = std::max(big, n.count);
      small = std::min(small, n.count);
    }
  info[0] = (int64_t)B.nodes.size();
  info[1] = leaves;
  info[2] = B.depth;
  info[3] = big;
  info[4] = small;
  info[5] = (int64_t)B.prims.size();
  return 0;
}

// Binary tree in neutral form: node i has children child[2i], child[2i+1]
// (>= 0 internal node index, < 0 leaf -1-l); leaf l covers
// prims[leaf_first[l] .. + leaf_count[l]).  Root is node 0, or leaf 0 when
// there is no internal node.  Arrays sized by orc_bvh_info.
int orc_bvh_export(void* h, int32_t* child, int64_t* leaf_first, int64_t* leaf_count,
                   int32_t* prims) {
  const Bvh& B = *static_cast<Bvh*>(h);
  std::vector<int32_t> internal_id(B.nodes.size(), -1), leaf_id(B.nodes.size(), -1);
  int32_t ni = 0, nl = 0;
  for (size_t i = 0; i < B.nodes.size(); ++i) {
    if (B.nodes[i].child[0] >= 0)
      internal_id[i] = ni++;
    else
      leaf_id[i] = nl++;
  }
  for (size_t i = 0; i < B.nodes.size(); ++i) {
    const Node& n = B.nodes[i];
    if (n.child[0] >= 0) {
      for (int s = 0; s < 2; ++s) {
        int32_t c = n.child[s];
        child[2 * internal_id[i] + s] = internal_id[c] >= 0 ? internal_id[c] : -1 - leaf_id[c];
      }
    } else {
      leaf_first[leaf_id[i]] = n.first;
      leaf_count[leaf_id[i]] = n.count;
    }
  }
  std::memcpy(prims, B.prims.data(), B.prims.size() * sizeof(int32_t));
  return 0;
}

int orc_bvh_closest(void* h, const float* rays, int64_t n_ray, const int32_t* skip, double* t_out,
                    int32_t* id_out, double* u_out, double* v_out, double* t2_out, int n_threads) {
  const Bvh& B = *static_cast<Bvh*>(h);
  parallel_for(n_ray, n_threads, [&](int64_t ri) {
    Ray r = load_ray(rays, ri);
    Best best;
    walk_closest(B, r, skip ? skip[ri] : -1, &best);
    t_out[ri] = best.t;
    id_out[ri] = best.id;
    if (u_out) u_out[ri] = best.u;
    if (v_out) v_out[ri] = best.v;
    if (t2_out) t2_out[ri] = best.t2;
  });
  return 0;
}

int orc_bvh_any(void* h, const float* rays, int64_t n_ray, const int32_t* skip, uint8_t* out,
                int n_threads) {
  const Bvh& B = *static_cast<Bvh*>(h);
  parallel_for(n_ray, n_threads, [&](int64_t ri) {
    Ray r = load_ray(rays, ri);
    out[ri] = walk_any(B, r, skip ? skip[ri] : -1) ? 1 : 0;
  });
  return 0;
}

// Eq. 2 for explicit boxes (lo[3], hi[3] each) and counts.
double orc_eq2_cost(const double* boxA, double kA, const double* boxB, double kB,
                    const double* boxC, double alpha, double t_i, double t_trav,
                    const double* source3, int dist_norm) {
  Box A, B, C;
  for (int a = 0; a < 3; ++a) {
    A.lo[a] = boxA[a];
    A.hi[a] = boxA[3 + a];
    B.lo[a] = boxB[a];
    B.hi[a] = boxB[3 + a];
    C.lo[a] = boxC[a];
    C.hi[a] = boxC[3 + a];
  }
  CostParams p{alpha, t_i, t_trav, {source3[0], source3[1], source3[2]}, dist_norm};
  return eq2(A, kA, B, kB, C, p);
}

// 5. Eq. 2 applied recursively to a binary tree in the neutral form of
// orc_bvh_export: cost(leaf) = k t_i; cost(C) = alpha (S(A)/S(C) cost(A) +
// S(B)/S(C) cost(B)) + (1 - alpha) d^2(A, B) + t_trav.  Boxes are recomputed
// from the triangles.  Returns NaN when the tree is malformed.
double orc_tree_cost(const float* tris, int64_t n_tri, int64_t n_internal, const int32_t* child,
                     const int64_t* leaf_first, const int64_t* leaf_count, int64_t n_leaves,
                     const int32_t* prims, double alpha, double t_i, double t_trav,
                     const double* source3, int dist_norm) {
  CostParams p{alpha, t_i, t_trav, {source3[0], source3[1], source3[2]}, dist_norm};
  auto leaf_box = [&](int64_t l, Box* b) {
    for (int64_t k = leaf_first[l]; k < leaf_first[l] + leaf_count[l]; ++k) {
      if (prims[k] < 0 || prims[k] >= n_tri) return false;
      b->add(tri_box(tris, prims[k]));
    }
    return true;
  };
  if (n_internal == 0) return n_leaves == 1 ? (double)leaf_count[0] * t_i : NAN;
  // post-order over internal nodes with an explicit stack
  std::vector<double> cost(n_internal, NAN), count(n_internal, 0.0);
  std::vector<Box> box(n_internal);
  std::vector<int8_t> state(n_internal, 0);
  std::vector<int32_t> st{0};
  int64_t guard = 0;
  while (!st.empty()) {
    if (++guard > 4 * (n_internal + 1)) return NAN;
    int32_t i = st.back();
    if (i < 0 || i >= n_internal) return NAN;
    if (state[i] == 0) {
      state[i] = 1;
      for (int s = 0; s < 2; ++s)
        if (child[2 * i + s] >= 0) st.push_back(child[2 * i + s]);
      continue;
    }
    st.pop_back();
    Box cb[2];
    double cc[2], kk[2];
    for (int s = 0; s < 2; ++s) {
      int32_t c = child[2 * i + s];
      if (c >= 0) {
        cb[s] = box[c];
        cc[s] = cost[c];
        kk[s] = count[c];
      } else {
        int64_t l = -1 - (int64_t)c;
        if (l >= n_leaves || !leaf_box(l, &cb[s])) return NAN;
        cc[s] = (double)leaf_count[l] * t_i;
        kk[s] = (double)leaf_count[l];
      }
    }
    Box C = cb[0];
    C.add(cb[1]);
    // Eq. 2 with the children's expected costs in place of k t_i
    double sc = C.area();
    double sah = sc > 0.0 ? (cb[0].area() / sc) * cc[0] + (cb[1].area() / sc) * cc[1] : cc[0] + cc[1];
    double dA2 = 0.0, dB2 = 0.0, diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      double ca = 0.5 * (cb[0].lo[a] + cb[0].hi[a]) - p.src[a];
      double cbb = 0.5 * (cb[1].lo[a] + cb[1].hi[a]) - p.src[a];
      double dc = C.hi[a] - C.lo[a];
      dA2 += ca * ca;
      dB2 += cbb * cbb;
      diag2 += dc * dc;
    }
    double d2 = 0.5 * (dA2 + dB2);
    if (p.dist_norm == 2)
      d2 = (diag2 > 0.0 ? (kk[0] * dA2 + kk[1] * dB2) / diag2 : 0.0) * p.t_i;
    else if (p.dist_norm)
      d2 = (diag2 > 0.0 ? d2 / diag2 : 0.0) * (kk[0] + kk[1]) * p.t_i;
    cost[i] = p.alpha * sah + (1.0 - p.alpha) * d2 + p.t_trav;
    count[i] = kk[0] + kk[1];
    box[i] = C;
  }
  return cost[0];
}

// 6. Specular reflection (Sec. III.B) of rays at their hits, float64.
// out8[r] = (o + t d, 0, d - 2 (d.n) n, tmax - t) with n the unit normal of
// (v1 - v0) x (v2 - v0).  Rays without a hit (id < 0) get tmax = -inf.
int orc_reflect(const float* tris, const float* rays, const int32_t* hit_id, const double* hit_t,
                int64_t n, double* out8) {
  for (int64_t ri = 0; ri < n; ++ri) {
    Ray r = load_ray(rays, ri);
    double* o = out8 + ri * 8;
    int32_t id = hit_id[ri];
    if (id < 0) {
      for (int k = 0; k < 8; ++k) o[k] = 0.0;
      o[7] = -kInf;
      continue;
    }
    double t = hit_t[ri];
    V3 nrm = cross(sub(vert(tris, id, 1), vert(tris, id, 0)), sub(vert(tris, id, 2), vert(tris, id, 0)));
    double len = std::sqrt(dot(nrm, nrm));
    nrm = {nrm.x / len, nrm.y / len, nrm.z / len};
    double dn = dot(r.d, nrm);
    o[0] = r.o.x + t * r.d.x;
    o[1] = r.o.y + t * r.d.y;
    o[2] = r.o.z + t * r.d.z;
    o[3] = 0.0;
    o[4] = r.d.x - 2.0 * dn * nrm.x;
    o[5] = r.d.y - 2.0 * dn * nrm.y;
    o[6] = r.d.z - 2.0 * dn * nrm.z;
    o[7] = r.tmax - t;
  }
  return 0;
}

// 7a. Fibonacci sphere: z_i = 1 - (2i+1)/n, azimuth i pi (3 - sqrt 5).
int orc_fibonacci(int64_t n, double* out3) {
  const double ga = M_PI * (3.0 - std::sqrt(5.0));
  for (int64_t i = 0; i < n; ++i) {
    double z = 1.0 - (2.0 * (double)i + 1.0) / (double)n;
    double rho = std::sqrt(std::max(0.0, 1.0 - z * z));
    double ph = (double)i * ga;
    out3[3 * i + 0] = rho * std::cos(ph);
    out3[3 * i + 1] = rho * std::sin(ph);
    out3[3 * i + 2] = z;
  }
  return 0;
}

// 7b. Icosahedral launch (Sec. III.A): the 12 vertices of a regular
// icosahedron, each of its 20 faces subdivided into f*f triangles
// (f = 2^level), directions to the distinct grid vertices, unit length.
// Returns the count (10 f^2 + 2); writes directions when out3 != NULL, in
// the order: corners, edge points (edges in lexicographic order, from the
// lower to the higher vertex index), face-interior points (faces in
// lexicographic order, grid index i outer, j inner).
int64_t orc_icosphere(int level, double* out3) {
  const int64_t f = (int64_t)1 << level;
  const int64_t count = 10 * f * f + 2;
  if (!out3) return count;
  const double g = (1.0 + std::sqrt(5.0)) / 2.0;
  std::vector<V3> v;
  for (double a : {-1.0, 1.0})
    for (double b : {-g, g}) {
      v.push_back({0.0, a, b});
      v.push_back({a, b, 0.0});
      v.push_back({b, 0.0, a});
    }
  const int nv = (int)v.size();
  auto adjacent = [&](int i, int j) {
    V3 d = sub(v[i], v[j]);
    return std::fabs(std::sqrt(dot(d, d)) - 2.0) < 1e-9;
  };
  std::vector<std::array<int, 3>> faces;
  std::vector<std::array<int, 2>> edges;
  for (int i = 0; i < nv; ++i)
    for (int j = i + 1; j < nv; ++j) {
      if (!adjacent(i, j)) continue;
      edges.push_back({i, j});
      for (int k = j + 1; k < nv; ++k)
        if (adjacent(j, k) && adjacent(i, k)) faces.push_back({i, j, k});
    }
  int64_t w = 0;
  auto emit = [&](V3 p) {
    double len = std::sqrt(dot(p, p));
    out3[3 * w + 0] = p.x / len;
    out3[3 * w + 1] = p.y / len;
    out3[3 * w + 2] = p.z / len;
    ++w;
  };
  for (const V3& p : v) emit(p);
  const double fd = (double)f;
  for (auto& e : edges)
    for (int64_t k = 1; k < f; ++k) {
      double s = (double)k / fd;
      V3 a = v[e[0]], b = v[e[1]];
      emit({a.x * (1.0 - s) + b.x * s, a.y * (1.0 - s) + b.y * s, a.z * (1.0 - s) + b.z * s});
    }
  for (auto& fc : faces)
    for (int64_t i = 1; i < f; ++i)
      for (int64_t j = 1; j < f - i; ++j) {
        double wi = (double)i / fd, wj = (double)j / fd, w0 = 1.0 - wi - wj;
        V3 a = v[fc[0]], b = v[fc[1]], c = v[fc[2]];
        emit({a.x * w0 + b.x * wi + c.x * wj, a.y * w0 + b.y * wi + c.y * wj,
              a.z * w0 + b.z * wi + c.z * wj});
      }
  return w;
}

// 8. Reception (Sec. III.C, Eq. 4), every ray segment against every
// receiver.  rays: float32 [n][8] (o, tmin, d, tmax); hit_t: float32 [n]
// (+inf: no hit); rx: float32 [m][3].  A pair is reported when it is
// received (class 1: inside by more than tol in distance to the sphere and
// in t* to both segment ends) or within tol of the boundary (class 2); pairs
// farther outside are not reported.  out_i: [cap][3] (ray, rx, class);
// out_d: [cap][3] (l, distance, radius).  Returns the number of pairs found
// (only the first cap are written).
int64_t orc_receive(const float* rays, const float* hit_t, int64_t n, const float* rx, int64_t m,
                    double delta, double range0, double tol, int32_t* out_i, double* out_d,
                    int64_t cap) {
  const double k = delta / std::sqrt(3.0);
  int64_t w = 0;
  for (int64_t i = 0; i < n; ++i) {
    const float* r = rays + 8 * i;
    const V3 o = {(double)r[0], (double)r[1], (double)r[2]};
    const V3 d = {(double)r[4], (double)r[5], (double)r[6]};
    const double tmin = (double)r[3], tmax = (double)r[7];
    const double th = (double)hit_t[i];
    const double tend = th < tmax ? th : tmax;
    const double dd = dot(d, d);
    if (!(dd > 0.0) || !(tend > tmin)) continue;
    const double lprev = range0 - tmax;
    for (int64_t j = 0; j < m; ++j) {
      const V3 p = {(double)rx[3 * j], (double)rx[3 * j + 1], (double)rx[3 * j + 2]};
      const V3 q = sub(p, o);
      const double ts = dot(q, d) / dd;
      const V3 f = {o.x + ts * d.x, o.y + ts * d.y, o.z + ts * d.z};
      const V3 e = sub(p, f);
      const double dist = std::sqrt(dot(e, e));
      const double l = lprev + ts;
      const double rad = l * k;
      // signed margins: positive inside
      const double mr = rad - dist, m0 = ts - tmin, m1 = tend - ts;
      const double lo = std::min(mr, std::min(m0, m1));
      if (lo < -tol) continue;
      if (w < cap) {
        out_i[3 * w] = (int32_t)i;
        out_i[3 * w + 1] = (int32_t)j;
        out_i[3 * w + 2] = lo > tol ? 1 : 2;
        out_d[3 * w] = l;
        out_d[3 * w + 1] = dist;
        out_d[3 * w + 2] = rad;
      }
      ++w;
    }
  }
  return w;
}

}  // extern "C"
