// Ray casting along multipath routes and per-hit backscatter (Sec. II.A-II.B).
//
// One thread traces one sub-ray of one ping through the whole route: closest hit by
// BVH traversal, optional specular continuation off mirror triangles and the sea
// surface (limited secondary reflections, maximum depth max_bounces), and, for every
// scattering hit, the FP64 two-way delay, the carrier phase reduced modulo one cycle,
// the Lambertian amplitude and the hashed speckle phase. Rays bend in a linear
// sound-speed profile as exact circular arcs intersected chord by chord.
//
// Precision: the traversal culls in FP32 with widened boxes and a slack barycentric
// test. A triangle whose FP32 barycentrics lie inside by more than the slack is a hit
// in FP64 too; every other survivor (near an edge, nearly parallel, near an interval
// end) is decided by an FP64 ray/triangle test written with explicitly rounded
// operations, and competing hits closer than the FP32 distance error are ordered by
// their FP64 distances. The distance of the chosen hit is always FP64 (from the
// stored FP64 plane), so delays and carrier phase keep FP64 accuracy. FP64 operations
// are scarce on this part: decisions (the ray/triangle test) use explicitly rounded
// operations in the oracle's order, while positions, distances and delays contract into
// FMAs (an ulp or so from the oracle), and amplitudes are FP32.
#include "common.cuh"

namespace sonar {
namespace {

// ----------------------------------------------------------------- FP64, no contraction
__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }

struct D3 { double x, y, z; };
__device__ __forceinline__ D3 d3(double x, double y, double z) { D3 r = {x, y, z}; return r; }
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return d3(ds(a.x, b.x), ds(a.y, b.y), ds(a.z, b.z)); }
__device__ __forceinline__ double dot(D3 a, D3 b) { return da(da(dm(a.x, b.x), dm(a.y, b.y)), dm(a.z, b.z)); }
// contracted forms for positions and distances
__device__ __forceinline__ double dotf(D3 a, D3 b) { return fma(a.z, b.z, fma(a.y, b.y, a.x * b.x)); }
__device__ __forceinline__ D3 rot(const double* R, D3 v) {
  return d3(fma(R[2], v.z, fma(R[1], v.y, R[0] * v.x)), fma(R[5], v.z, fma(R[4], v.y, R[3] * v.x)),
            fma(R[8], v.z, fma(R[7], v.y, R[6] * v.x)));
}
__device__ __forceinline__ D3 rot_t(const double* R, D3 v) {
  return d3(da(da(dm(R[0], v.x), dm(R[3], v.y)), dm(R[6], v.z)),
            da(da(dm(R[1], v.x), dm(R[4], v.y)), dm(R[7], v.z)),
            da(da(dm(R[2], v.x), dm(R[5], v.y)), dm(R[8], v.z)));
}

// a / b for |b| in [1e-30, 1e30]: an FP32 reciprocal seed refined by one Newton-Raphson
// step y += y (1 - b y) (relative error 2^-23 -> 2^-46), then one residual correction of
// the quotient q += (a - b q) y, which squares the error again (to rounding level).
// Within an ulp or so of the correctly rounded quotient at a fraction of the cost of
// FP64 division, which is long on this part.
__device__ __forceinline__ double ddiv_nr(double a, double b) {
  double y = (double)__frcp_rn((float)b);
  y = fma(y, fma(-b, y, 1.0), y);
  const double q = a * y;
  return fma(fma(-b, q, a), y, q);
}
// 1 / sqrt(s) for s in [1e-30, 1e30]: FP32 seed, two Newton-Raphson steps
// y *= (3 - s y^2) / 2.
__device__ __forceinline__ double drsqrt_nr(double s) {
  double y = (double)rsqrtf((float)s);
  y = y * fma(-0.5 * s, y * y, 1.5);
  y = y * fma(-0.5 * s, y * y, 1.5);
  return y;
}

// ----------------------------------------------------------------- FP32 pairs
// A value as the unevaluated sum hi + lo of two FP32 numbers, |lo| <= ulp(hi) / 2, about
// 48 significant bits: Dekker's double-length arithmetic (Dekker 1971), with Knuth's
// error-free sum and the FMA product error. FP32 issues at many times the FP64 rate on
// this part, so the straight-ray path carries its geometry, delays and phases in pairs:
// ~2^-46 relative per operation against the 1e-12 the delays need. The explicitly rounded
// operations keep the compiler from contracting the error terms away.
struct F2 {
  float hi, lo;
};
struct DF3 {
  F2 x, y, z;
};
__device__ __forceinline__ F2 f2(float a) { return F2{a, 0.f}; }
__device__ __forceinline__ F2 f2(float2 v) { return F2{v.x, v.y}; }
__device__ __forceinline__ F2 quick_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return F2{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ F2 operator+(F2 x, F2 y) {
  F2 s = two_sum(x.hi, y.hi);
  const F2 t = two_sum(x.lo, y.lo);
  s = quick_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return quick_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ F2 operator-(F2 x) { return F2{-x.hi, -x.lo}; }
__device__ __forceinline__ F2 operator-(F2 x, F2 y) { return x + (-y); }
__device__ __forceinline__ F2 operator*(F2 x, F2 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return quick_two_sum(p, e);
}
// x / y by long division: three quotient digits from one FP32 reciprocal of y.hi, each
// taken from the remainder the previous ones leave.
__device__ __forceinline__ F2 operator/(F2 x, F2 y) {
  const float r = __frcp_rn(y.hi);
  const float q1 = __fmul_rn(x.hi, r);
  F2 rem = x - f2(q1) * y;
  const float q2 = __fmul_rn(rem.hi, r);
  rem = rem - f2(q2) * y;
  const float q3 = __fmul_rn(rem.hi, r);
  return quick_two_sum(q1, q2) + f2(q3);
}
// pairs are normalised (hi = RN(hi + lo)), so these compare values
__device__ __forceinline__ bool operator<(F2 a, F2 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator==(F2 a, F2 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ F2 dot(const DF3& a, const DF3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ DF3 axpy(const DF3& p, F2 t, const DF3& d) {
  return DF3{p.x + t * d.x, p.y + t * d.y, p.z + t * d.z};
}
// sqrt of a pair: the FP32 root s of hi, then one Newton correction from the exact
// residual v - s^2 (s^2 as an error-free product)
__device__ __forceinline__ F2 sqrt_df(F2 v) {
  const float s = __fsqrt_rn(v.hi);
  if (!(s > 0.f)) return F2{s, 0.f};
  const float p = __fmul_rn(s, s);
  const F2 r = v - F2{p, __fmaf_rn(s, s, -p)};
  return quick_two_sum(s, __fdiv_rn(r.hi, __fmul_rn(2.f, s)));
}
// FP64 views, for the FP64 legs' geometry and the debug delays
__device__ __forceinline__ double to_d(F2 v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ D3 to_d3(const DF3& v) { return d3(to_d(v.x), to_d(v.y), to_d(v.z)); }
__device__ __forceinline__ F2 f2_of(double x) {
  const float hi = (float)x;
  return F2{hi, (float)(x - (double)hi)};
}


__device__ __forceinline__ double4_32a load_plane(const DevScene& sc, int leaf) {
  const double2* p = reinterpret_cast<const double2*>(sc.tri_plane + leaf);
  const double2 a = __ldg(p), b = __ldg(p + 1);
  return make_double4_32a(a.x, a.y, b.x, b.y);
}

// |cos| of the incidence angle from the stored FP64 plane normal: the dot product in
// FP64 (grazing incidence keeps its relative accuracy), the scaling in FP32.
__device__ __forceinline__ float kinc32(const DevScene& sc, int leaf, D3 d) {
  const double4_32a P = load_plane(sc, leaf);
  return fabsf((float)dotf(d, d3(P.x, P.y, P.z))) * __ldg(&sc.tri_inv_n[leaf]);
}

// Unit geometric normal (b - a) x (c - a) / |.| in FP64, for specular reflection.
__device__ D3 tri_normal64(const DevScene& sc, int leaf) {
  const double4_32a P = load_plane(sc, leaf);
  const D3 n = d3(P.x, P.y, P.z);
  const double il = drsqrt_nr(dotf(n, n));
  return d3(dm(n.x, il), dm(n.y, il), dm(n.z, il));
}

__device__ __forceinline__ DF3 plane_n_df(const DevScene& sc, int leaf, F2& w) {
  const float4 h = __ldg(&sc.tri_plane_df[2 * leaf]), l = __ldg(&sc.tri_plane_df[2 * leaf + 1]);
  w = F2{h.w, l.w};
  return DF3{F2{h.x, l.x}, F2{h.y, l.y}, F2{h.z, l.z}};
}
__device__ __forceinline__ float kinc32(const DevScene& sc, int leaf, const DF3& d) {
  F2 w;
  const DF3 n = plane_n_df(sc, leaf, w);
  return fabsf(dot(d, n).hi) * __ldg(&sc.tri_inv_n[leaf]);
}

// ----------------------------------------------------------------- traversal
struct Ray32 {
  float ox, oy, oz, ix, iy, iz, dx, dy, dz;
};

__device__ __forceinline__ void slab(float lox, float hix, float loy, float hiy, float loz, float hiz,
                                     const Ray32& r, float tlo, float thi, float& tn, float& tf) {
  float x0 = (lox - r.ox) * r.ix, x1 = (hix - r.ox) * r.ix;
  float y0 = (loy - r.oy) * r.iy, y1 = (hiy - r.oy) * r.iy;
  float z0 = (loz - r.oz) * r.iz, z1 = (hiz - r.oz) * r.iz;
  tn = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), tlo));
  tf = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), thi));
}

template <class R>
struct HitT {
  R t;
  int prim;  // original id, -1 none
  int leaf;
};
using Hit = HitT<double>;

// FP64 distance to the triangle's plane: (n . a - n . o) / (n . d).
__device__ __forceinline__ double plane_t(const DevScene& sc, int leaf, D3 o, D3 d) {
  const double4_32a P = load_plane(sc, leaf);
  const D3 n = d3(P.x, P.y, P.z);
  return ddiv_nr(P.w - dotf(n, o), dotf(n, d));
}
// The same from the plane's FP32 pairs.
__device__ __forceinline__ F2 plane_t(const DevScene& sc, int leaf, const DF3& o, const DF3& d) {
  F2 w;
  const DF3 n = plane_n_df(sc, leaf, w);
  return (w - dot(n, o)) / dot(n, d);
}

// Generic pieces of the traversal over the two precisions of its exact parts.
__device__ __forceinline__ float to_f(double x) { return (float)x; }
__device__ __forceinline__ float to_f(F2 x) { return x.hi; }
__device__ __forceinline__ void lead32(const D3& v, float* f) { f[0] = (float)v.x; f[1] = (float)v.y; f[2] = (float)v.z; }
__device__ __forceinline__ void lead32(const DF3& v, float* f) { f[0] = v.x.hi; f[1] = v.y.hi; f[2] = v.z.hi; }
__device__ __forceinline__ void r_inf(double& x) { x = INFINITY; }
__device__ __forceinline__ void r_inf(F2& x) { x = F2{INFINITY, 0.f}; }
// Near-tie ray/triangle decision with its distance inside (tmin, tmax], for the FP64
// legs (curved rays, field routes, point, cross-term and volume legs): the FP32-pair test
// below, whose decision differs from an FP64 one only for margins below ~1e-13.
__device__ bool tri_test_df(const float* tv, const struct DF3& o, const struct DF3& d, F2& t);
__device__ __forceinline__ bool tri_exact(const float* tv, const D3& o, const D3& d, double tmin, double tmax,
                                          double& t) {
  F2 tp;
  if (!tri_test_df(tv, DF3{f2_of(o.x), f2_of(o.y), f2_of(o.z)}, DF3{f2_of(d.x), f2_of(d.y), f2_of(d.z)}, tp))
    return false;
  t = to_d(tp);
  return t > tmin && t <= tmax;
}
// The same two-sided test in FP32 pairs (edges exact from the FP32 vertices; ~2^-46
// relative after that). Its decision differs from an FP64 test's only where u, v or
// 1 - u - v lies within ~1e-13 of zero, far inside the barycentric margin (1e-5) outside
// which hits must agree; it keeps the straight-ray and volume paths off the FP64 pipe,
// which issues at a small fraction of the FP32 rate on this part and was a third busy
// with these tests alone.
__device__ __forceinline__ DF3 cross_df(const DF3& a, const DF3& b) {
  return DF3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ bool tri_test_df(const float* tv, const DF3& o, const DF3& d, F2& t) {
  const DF3 e1 = DF3{two_sum(tv[3], -tv[0]), two_sum(tv[4], -tv[1]), two_sum(tv[5], -tv[2])};
  const DF3 e2 = DF3{two_sum(tv[6], -tv[0]), two_sum(tv[7], -tv[1]), two_sum(tv[8], -tv[2])};
  const DF3 p = cross_df(d, e2);
  const F2 det = dot(e1, p);
  if (!(fabsf(det.hi) > 1e-30f)) return false;
  const F2 inv = f2(1.f) / det;
  const DF3 s = DF3{o.x - f2(tv[0]), o.y - f2(tv[1]), o.z - f2(tv[2])};
  const F2 u = dot(s, p) * inv;
  if (u < f2(0.f) || f2(1.f) < u) return false;
  const DF3 q = cross_df(s, e1);
  const F2 v = dot(d, q) * inv;
  if (v < f2(0.f) || f2(1.f) < u + v) return false;
  t = dot(e2, q) * inv;
  return true;
}
__device__ __forceinline__ bool tri_exact(const float* tv, const DF3& o, const DF3& d, F2 tmin, F2 tmax, F2& t) {
  if (!tri_test_df(tv, o, d, t)) return false;
  return tmin < t && !(tmax < t);
}

// Per-ray state of a closest-hit query: the ray in FP32 for the filter tests, the
// interval, the cull distance and the best hit so far.
template <class R>
struct HitQuery {
  Ray32 r;
  float tmin32, tmax32, tcull;
  HitT<R> best;
  bool best_exact;
  float best_t32;
};

template <class V, class R>
__device__ __forceinline__ void query_init(HitQuery<R>& q, const V& o, const V& d, R tmin, R tmax, const float* o32,
                                           const float* d32) {
  r_inf(q.best.t);
  q.best.prim = -1;
  q.best.leaf = -1;
  q.best_exact = true;
  q.best_t32 = INFINITY;
  float f[3];
  if (o32) {
    q.r.ox = o32[0]; q.r.oy = o32[1]; q.r.oz = o32[2];
  } else {
    lead32(o, f);
    q.r.ox = f[0]; q.r.oy = f[1]; q.r.oz = f[2];
  }
  if (d32) {
    q.r.dx = d32[0]; q.r.dy = d32[1]; q.r.dz = d32[2];
  } else {
    lead32(d, f);
    q.r.dx = f[0]; q.r.dy = f[1]; q.r.dz = f[2];
  }
  q.r.ix = __frcp_rn(q.r.dx); q.r.iy = __frcp_rn(q.r.dy); q.r.iz = __frcp_rn(q.r.dz);
  q.tmin32 = to_f(tmin);  // the loop stays in FP32
  q.tmax32 = to_f(tmax);
  q.tcull = to_f(tmax) * (1.0f + 1e-6f) + 1e-4f;
}

// One leaf candidate of a closest-hit query: the FP32 slack filter, the exact test where
// the filter cannot decide, and the comparison with the best hit (ties to the lowest
// primitive id). Returns true when ANY is set and the candidate is confirmed.
template <class V, class R, bool ANY>
__device__ __forceinline__ bool leaf_candidate(const DevScene& sc, HitQuery<R>& q, const V& o, const V& d, R tmin,
                                               R tmax, int exclude, int leaf) {
  const Ray32& r = q.r;
  float4 v0 = __ldg(&sc.tri32[3 * leaf]), e1 = __ldg(&sc.tri32[3 * leaf + 1]), e2 = __ldg(&sc.tri32[3 * leaf + 2]);
  float px = r.dy * e2.z - r.dz * e2.y, py = r.dz * e2.x - r.dx * e2.z, pz = r.dx * e2.y - r.dy * e2.x;
  float det = e1.x * px + e1.y * py + e1.z * pz;
  float n1 = e1.x * e1.x + e1.y * e1.y + e1.z * e1.z, n2 = e2.x * e2.x + e2.y * e2.y + e2.z * e2.z;
  bool pass, in32 = false;
  float t32 = 0.f;
  if (det * det <= 1e-12f * n1 * n2) {
    pass = true;  // nearly parallel: let FP64 decide
  } else {
    float inv = 1.0f / det;
    float sx = r.ox - v0.x, sy = r.oy - v0.y, sz = r.oz - v0.z;
    float u = (sx * px + sy * py + sz * pz) * inv;
    float qx = sy * e1.z - sz * e1.y, qy = sz * e1.x - sx * e1.z, qz = sx * e1.y - sy * e1.x;
    float v = (r.dx * qx + r.dy * qy + r.dz * qz) * inv;
    t32 = (e2.x * qx + e2.y * qy + e2.z * qz) * inv;
    float eps = 1e-3f + 1e-5f * sqrtf(n1 * n2 / (det * det)) * (1.0f + fabsf(t32));
    pass = u >= -eps && v >= -eps && u + v <= 1.0f + eps && t32 <= q.tcull && t32 >= -1e-3f;
    in32 = u >= eps && v >= eps && u + v <= 1.0f - eps;
  }
  if (!pass) return false;
  int prim = __ldg(&sc.tri_prim[leaf]);
  if (prim == exclude) return false;
  // A candidate is definite when its FP32 barycentrics are inside by more than the
  // slack and its distance clears both interval ends: FP64 would accept it too, so
  // only its distance is needed, and only when it competes with another hit.
  const float tslack = 1e-4f + 1e-5f * fabsf(t32);
  const bool definite = in32 && t32 >= q.tmin32 + tslack && t32 <= q.tmax32 - tslack;
  R t64;
  r_inf(t64);
  bool exact = false;
  if (!definite) {
    if (!tri_exact(sc.triv + 9 * leaf, o, d, tmin, tmax, t64)) return false;
    exact = true;
  }
  if (ANY) {
    q.best.prim = prim;
    q.best.leaf = leaf;
    return true;
  }
  bool take;
  if (q.best.prim < 0) {
    take = true;
  } else if (!exact && t32 < q.best_t32 - tslack) {
    take = true;
  } else if (!exact && t32 > q.best_t32 + tslack) {
    take = false;
  } else {
    // close or exact: compare FP64 distances, ties to the lowest primitive id
    if (!exact) { t64 = plane_t(sc, leaf, o, d); exact = true; }
    if (!q.best_exact) { q.best.t = plane_t(sc, q.best.leaf, o, d); q.best_exact = true; }
    take = t64 < q.best.t || (t64 == q.best.t && prim < q.best.prim);
  }
  if (take) {
    q.best.prim = prim;
    q.best.leaf = leaf;
    q.best.t = t64;
    q.best_exact = exact;
    q.best_t32 = exact ? to_f(t64) : t32;
    q.tcull = fminf(q.tcull, q.best_t32 * (1.0f + 1e-5f) + 2e-4f);
  }
  return false;
}

template <class V, class R>
__device__ __forceinline__ HitT<R> query_result(const DevScene& sc, HitQuery<R>& q, const V& o, const V& d) {
  if (q.best.prim >= 0 && !q.best_exact) q.best.t = plane_t(sc, q.best.leaf, o, d);
  return q.best;
}

// Nearest triangle with FP64 distance in (tmin, tmax], excluding `exclude` (original
// id), ties to the lowest id. The distance of the returned hit is FP64.
// o32, d32: the origin and the direction in FP32 when the caller has them (nullptr:
// converted here). An FP32 direction from FP32 operands differs from the FP64 one by
// ~1e-7, far inside the traversal's slack.
// ANY: an existence query (shadow legs): it returns the first triangle confirmed inside
// the interval, whose distance it leaves unset.
template <class V, class R, bool ANY = false>
__device__ HitT<R> closest_hit(const DevScene& sc, const V& o, const V& d, R tmin, R tmax, int exclude, int* err,
                               const float* o32 = nullptr, const float* d32 = nullptr) {
  HitQuery<R> q;
  query_init(q, o, d, tmin, tmax, o32, d32);
  if (sc.n_tris == 0) return q.best;
  int stack[kMaxStack];
  int sp = 0;
  int node = sc.root;
  const int max_visits = 2 * sc.n_tris + 64;  // a tree visits each node at most once
  for (int visits = 0;; ++visits) {
    if (visits > max_visits) { atomicOr(err, kErrLoop); break; }
    const BvhNode* nd = sc.nodes + node;
    float4 A = __ldg(&nd->a), B = __ldg(&nd->b), Cz = __ldg(&nd->c);
    int4 ch = __ldg(&nd->d);
    float ln, lf, rn, rf;
    slab(A.x, A.y, A.z, A.w, Cz.x, Cz.y, q.r, -1e-4f, q.tcull, ln, lf);
    slab(B.x, B.y, B.z, B.w, Cz.z, Cz.w, q.r, -1e-4f, q.tcull, rn, rf);
    bool hl = ln <= lf, hr = rn <= rf;
    // leaf children: one copy of the triangle test, run for each (a rolled loop keeps the
    // traversal loop small in the instruction cache)
    const bool leaf_l = hl && ch.x < 0, leaf_r = hr && ch.y < 0;
#pragma unroll 1
    for (int c = leaf_l ? 0 : 1; c < (leaf_r ? 2 : 1); ++c) {
      if (c == 0 || leaf_r)
        if (leaf_candidate<V, R, ANY>(sc, q, o, d, tmin, tmax, exclude, ~(c == 0 ? ch.x : ch.y))) return q.best;
    }
    hl = hl && !leaf_l;
    hr = hr && !leaf_r;
    if (hl && hr) {
      int nearc = ln <= rn ? ch.x : ch.y, farc = ln <= rn ? ch.y : ch.x;
      if (sp >= kMaxStack) { atomicOr(err, kErrStack); break; }
      stack[sp++] = farc;
      node = nearc;
    } else if (hl) {
      node = ch.x;
    } else if (hr) {
      node = ch.y;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
  return query_result(sc, q, o, d);
}

// Warp-cooperative closest hit, called by all 32 lanes of a warp together (lanes with
// live = false ride along). Every lane keeps its own ray, interval, cull distance and
// best hit; the warp walks one shared stack (wstack: kMaxStack ints of shared memory per
// warp) and visits a node when the ray of any live lane overlaps it, nearer child first
// by the lanes' majority. Node and triangle loads are broadcasts and the traversal loop
// does not diverge. Each lane's result is its own closest hit, ties to the lowest id,
// whatever the visit order: the cull distance never drops below a lane's best.
template <class V, class R>
__device__ HitT<R> closest_hit_warp(const DevScene& sc, const V& o, const V& d, R tmin, R tmax, int exclude, int* err,
                                    bool live, int* wstack, const float* o32 = nullptr) {
  HitQuery<R> q;
  query_init(q, o, d, tmin, tmax, o32, nullptr);
  const unsigned full = 0xffffffffu;
  if (sc.n_tris == 0 || !__any_sync(full, live)) return q.best;
  const int lane = threadIdx.x & 31;
  int sp = 0;
  int node = sc.root;
  const int max_visits = 2 * sc.n_tris + 64;
  for (int visits = 0;; ++visits) {
    if (visits > max_visits) {
      if (lane == 0) atomicOr(err, kErrLoop);
      break;
    }
    const BvhNode* nd = sc.nodes + node;
    float4 A = __ldg(&nd->a), B = __ldg(&nd->b), Cz = __ldg(&nd->c);
    int4 ch = __ldg(&nd->d);
    bool hl = false, hr = false;
    float ln = 0.f, rn = 0.f;
    if (live) {
      float lf, rf;
      slab(A.x, A.y, A.z, A.w, Cz.x, Cz.y, q.r, -1e-4f, q.tcull, ln, lf);
      slab(B.x, B.y, B.z, B.w, Cz.z, Cz.w, q.r, -1e-4f, q.tcull, rn, rf);
      hl = ln <= lf;
      hr = rn <= rf;
      if (hl && ch.x < 0) {
        hl = false;
        leaf_candidate<V, R, false>(sc, q, o, d, tmin, tmax, exclude, ~ch.x);
      }
      if (hr && ch.y < 0) {
        hr = false;
        leaf_candidate<V, R, false>(sc, q, o, d, tmin, tmax, exclude, ~ch.y);
      }
    }
    const bool any_l = __any_sync(full, hl), any_r = __any_sync(full, hr);
    if (any_l && any_r) {
      const int lfirst = __popc(__ballot_sync(full, hl && hr && ln <= rn));
      const int rfirst = __popc(__ballot_sync(full, hl && hr && ln > rn));
      const bool left_near = lfirst >= rfirst;
      if (sp >= kMaxStack) {
        if (lane == 0) atomicOr(err, kErrStack);
        break;
      }
      if (lane == 0) wstack[sp] = left_near ? ch.y : ch.x;
      ++sp;
      node = left_near ? ch.x : ch.y;
    } else if (any_l) {
      node = ch.x;
    } else if (any_r) {
      node = ch.y;
    } else {
      if (sp == 0) break;
      __syncwarp();
      node = wstack[--sp];
      __syncwarp();
    }
  }
  return query_result(sc, q, o, d);
}

// ----------------------------------------------------------------- hit emission
__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long* counter) {
  unsigned mask = __activemask();
  int lane = threadIdx.x & 31;
  int leader = __ffs(mask) - 1;
  unsigned rank = __popc(mask & ((1u << lane) - 1u));
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + rank;
}

// Counts a hit of first-tap row g (g < 0: no tap in range) into the histogram: one atomic
// per distinct row among the emitting lanes. With bin_rank the atomic's old count plus the
// lane's place among its row's lanes is the hit's rank in its row, so the counting sort
// scatters without atomics.
__device__ __forceinline__ void bin_count(const TraceArgs& A, int g, unsigned long long slot) {
  const unsigned act = __activemask();
  const unsigned grp = __match_any_sync(act, g);
  const int lane = (int)(threadIdx.x & 31), leader = __ffs(grp) - 1;
  if (!A.bin_rank) {
    if (g >= 0 && lane == leader) atomicAdd(&A.bin_counts[g], __popc(grp));
    return;
  }
  int base = 0;
  if (g >= 0 && lane == leader) base = atomicAdd(&A.bin_counts[g], __popc(grp));
  base = __shfl_sync(act, base, leader);
  if (g >= 0) A.bin_rank[slot] = base + __popc(grp & ((1u << lane) - 1u));
}

// tau: FP64 two-way delay; amp: |c_k|; psi_cyc: speckle phase in cycles; (uy, uz):
// sonar-frame arrival direction.
__device__ void emit(const TraceArgs& A, int ping, double tau, float amp, double psi_cyc, float uy, float uz,
                     int prim, uint32_t key) {
  unsigned long long slot = warp_reserve(A.n_hits);
  if ((int64_t)slot >= A.hit_cap) { atomicOr(A.err, kErrCapacity); return; }
  // phase psi - f0 tau in cycles, reduced modulo one cycle in FP64 to [-1/2, 1/2] before
  // forming the phasor
  double cyc = fma(-A.f0, tau, psi_cyc);
  cyc -= rint(cyc);
  // fractional sample position q = (tau - t0) / dt; first tap nf = floor(q - hw) + 1
  const double q = fma(tau, A.inv_dt, -A.t0_dt);
  const double nf = floor(q - A.hw) + 1.0;
  HitRec h;
  // a hit whose first tap lies outside this ping's padded rows has no tap in range
  const int64_t nfi = (int64_t)nf;  // saturating conversion; |nf| is bounded by T_stop anyway
  const bool in_rows = nfi >= -kPad && nfi < (int64_t)A.nr_pad - kPad;
  h.nglob = in_rows ? ping * A.nr_pad + (int)nfi + kPad : -1;
  h.u0 = (float)(nf - q);
  // histogram of first-tap rows for the counting sort: one atomic per distinct row among
  // the emitting lanes, whose old count places each lane's hit within its row
  bin_count(A, h.nglob, slot);
  float s, c;
  sincospif(2.0f * (float)cyc, &s, &c);
  h.cr = amp * c;
  h.ci = amp * s;
  h.uy = uy;
  h.uz = uz;
  h.prim = prim;
  h.key = key;
  A.hits[slot] = h;
  if (A.dbg_tau) A.dbg_tau[slot] = tau;
}

// Speckle phase of a hit in cycles: a 24-bit uniform fraction from the hash (exact in FP64).
// emit() for the straight-ray path, from a two-way delay held as an FP32 pair: the
// phase psi - f0 tau with f0 tau's integer part removed exactly, the sample position
// q = tau / dt - t0 / dt and its first tap floor(q - hw) + 1, all in pairs.
__device__ void emit_df(const TraceArgs& A, int ping, F2 tau, float amp, float psi_cyc, float uy, float uz,
                        int prim, uint32_t key) {
  unsigned long long slot = warp_reserve(A.n_hits);
  if ((int64_t)slot >= A.hit_cap) { atomicOr(A.err, kErrCapacity); return; }
  const F2 y = f2(psi_cyc) - f2(A.f0_df) * tau;
  const float k = rintf(y.hi);
  const float cyc = __fadd_rn(__fsub_rn(y.hi, k), y.lo);  // y.hi - k is exact
  const F2 q = tau * f2(A.inv_dt_df) - f2(A.t0_dt_df);
  const F2 z = q - f2(A.hw_df);
  float fl = floorf(z.hi);
  if (fl == z.hi && z.lo < 0.f) fl -= 1.f;  // an integral hi with a negative lo
  const float nf = fminf(fmaxf(fl + 1.f, -1e9f), 1e9f);
  HitRec h;
  const int nfi = (int)nf;
  const bool in_rows = nfi >= -kPad && nfi < A.nr_pad - kPad;
  h.nglob = in_rows ? ping * A.nr_pad + nfi + kPad : -1;
  h.u0 = __fsub_rn(__fsub_rn(nf, q.hi), q.lo);  // nf - q.hi is exact (Sterbenz)
  bin_count(A, h.nglob, slot);
  float s, c;
  sincospif(2.0f * cyc, &s, &c);
  h.cr = amp * c;
  h.ci = amp * s;
  h.uy = uy;
  h.uz = uz;
  h.prim = prim;
  h.key = key;
  A.hits[slot] = h;
  if (A.dbg_tau) A.dbg_tau[slot] = to_d(tau);
}

__device__ __forceinline__ double speckle(const TraceArgs& A, uint32_t ray, uint32_t sub, uint32_t bounce) {
  uint32_t x = ray, y = sub, z = 1u + bounce, w = A.seed32;
  pcg4d(x, y, z, w);
  return u24(x);
}
// the same in FP32 (a 24-bit fraction, exact in FP32)
__device__ __forceinline__ float speckle32(const TraceArgs& A, uint32_t ray, uint32_t sub, uint32_t bounce) {
  uint32_t x = ray, y = sub, z = 1u + bounce, w = A.seed32;
  pcg4d(x, y, z, w);
  return (float)(x >> 8) * (1.0f / 16777216.0f);
}

// Lambertian amplitude Gamma^2 sqrt(mu cos(k) dOmega) / L exp(-2 alpha L), in FP32: the
// amplitude needs no more than FP32 precision, unlike the delay and phase.
__device__ __forceinline__ float lambert(const TraceArgs& A, float gam, float mu, float kinc, float dOmega, float L) {
  return gam * gam * sqrtf(mu * kinc * dOmega) / L * expf(-2.0f * A.alpha32 * L);
}

// ----------------------------------------------------------------- curved rays
__device__ __forceinline__ double sincd(double x) { return fabs(x) < 1e-4 ? 1.0 - x * x / 6.0 : sin(x) / x; }

struct Arc {
  double dh, dz, theta, dt;
};
__device__ Arc arc_advance(const TraceArgs& A, double z, double theta, double xi, double step) {
  Arc r;
  double g = A.ssp_g;
  double delta = xi * g * step;
  double thm = theta - delta / 2;
  double sc = sincd(delta / 2);
  double cm = cos(thm);
  r.dh = step * cm * sc;
  r.dz = step * sin(thm) * sc;
  r.theta = theta - delta;
  if (fabs(cos(theta)) < 1e-12) {
    double c0 = A.ssp_c0 + g * (z - A.ssp_z0), c1 = A.ssp_c0 + g * (z + r.dz - A.ssp_z0);
    r.dt = g == 0.0 ? step / c0 : log(c1 / c0) / (g * sin(theta));
    return r;
  }
  double sh = sin(delta / 2);
  double xg = cm * xi * step * sc / (sh * sh + cm * cm);
  double x = g * xg;
  double ratio = fabs(x) < 1e-6 ? 1.0 + x * x / 3.0 : atanh(x) / x;
  r.dt = ratio * xg;
  return r;
}
__device__ __forceinline__ double arc_step(const TraceArgs& A, double xi) {
  double k = xi * fabs(A.ssp_g);
  if (k <= 0.0) return 2.0;
  return fmin(2.0, sqrt(8.0 / k * 1e-4));
}
__device__ __forceinline__ void dir_split(D3 d, double& ex, double& ey, double& theta) {
  double hz = sqrt(d.x * d.x + d.y * d.y);
  if (hz > 0) { ex = d.x / hz; ey = d.y / hz; } else { ex = 1.0; ey = 0.0; }
  theta = atan2(d.z, hz);
}
__device__ __forceinline__ double ssp_c(const TraceArgs& A, double z) { return A.ssp_c0 + A.ssp_g * (z - A.ssp_z0); }

// ----------------------------------------------------------------- 2-D sound-speed field
// Sec. II.A rays bent by a range- and depth-dependent sound speed. c(x, z) is bilinear
// on the grid, positions clamped to it (c constant outward, the gradient across a clamped
// axis zero); returns c and (dc/dx, dc/dz). FP64 division is a long instruction sequence
// on this part, so the grid spacings enter as host-computed reciprocals (results differ
// from divided ones by an ulp).
__device__ void field_eval(const TraceArgs& A, double x, double z, double& c, double& cx, double& cz) {
  const int nx = A.fld_nx, nz = A.fld_nz;
  double fx = (x - A.fld_x0) * A.fld_idx, fz = (z - A.fld_z0) * A.fld_idz;
  bool inx = true, inz = true;
  if (fx < 0.0) { fx = 0.0; inx = false; } else if (fx > nx - 1) { fx = nx - 1; inx = false; }
  if (fz < 0.0) { fz = 0.0; inz = false; } else if (fz > nz - 1) { fz = nz - 1; inz = false; }
  int i = (int)floor(fx), j = (int)floor(fz);
  if (i > nx - 2) i = nx - 2;
  if (j > nz - 2) j = nz - 2;
  const double u = fx - i, v = fz - j;
  const double* C = A.fld_c;
  const double c00 = __ldg(&C[j * nx + i]), c10 = __ldg(&C[j * nx + i + 1]);
  const double c01 = __ldg(&C[(j + 1) * nx + i]), c11 = __ldg(&C[(j + 1) * nx + i + 1]);
  c = (1.0 - u) * (1.0 - v) * c00 + u * (1.0 - v) * c10 + (1.0 - u) * v * c01 + u * v * c11;
  cx = inx ? ((1.0 - v) * (c10 - c00) + v * (c11 - c01)) * A.fld_idx : 0.0;
  cz = inz ? ((1.0 - u) * (c01 - c00) + u * (c11 - c10)) * A.fld_idz : 0.0;
}

// Ray equations in arc length for (r, t, T), t the unit tangent:
// dr/ds = t, dt/ds = ((grad c . t) t - grad c) / c, dT/ds = 1 / c.
__device__ __forceinline__ void field_deriv(const TraceArgs& A, const double (&y)[7], double (&f)[7]) {
  double c, cx, cz;
  field_eval(A, y[0], y[2], c, cx, cz);
  const double ic = ddiv_nr(1.0, c);  // one reciprocal (within an ulp of 1 / c)
  const double gt = cx * y[3] + cz * y[5];
  f[0] = y[3];
  f[1] = y[4];
  f[2] = y[5];
  f[3] = (gt * y[3] - cx) * ic;
  f[4] = gt * y[4] * ic;
  f[5] = (gt * y[5] - cz) * ic;
  f[6] = ic;
}

// One classical Runge-Kutta step of length h, the tangent renormalised after it.
__device__ void rk4_field(const TraceArgs& A, const double (&y)[7], double h, double (&out)[7]) {
  double k1[7], k2[7], k3[7], k4[7], tmp[7];
  field_deriv(A, y, k1);
#pragma unroll
  for (int i = 0; i < 7; ++i) tmp[i] = y[i] + 0.5 * h * k1[i];
  field_deriv(A, tmp, k2);
#pragma unroll
  for (int i = 0; i < 7; ++i) tmp[i] = y[i] + 0.5 * h * k2[i];
  field_deriv(A, tmp, k3);
#pragma unroll
  for (int i = 0; i < 7; ++i) tmp[i] = y[i] + h * k3[i];
  field_deriv(A, tmp, k4);
#pragma unroll
  for (int i = 0; i < 7; ++i) out[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  const double in = drsqrt_nr(out[3] * out[3] + out[4] * out[4] + out[5] * out[5]);
  out[3] *= in;
  out[4] *= in;
  out[5] *= in;
}

// Route in the field: RK4 steps of fld_h, the chord of each step intersected with the
// scene and the sea surface; a hit's time and arc length interpolate the step's end values
// in the chord fraction f; a reflection reflects the normalised (1 - f) t_i + f t_i+1.
__device__ void route_field(const TraceArgs& A, int ping, D3 o, D3 d0, D3 us, uint32_t ray, uint32_t sub,
                            double dOmega, uint32_t keybase) {
  double y[7] = {o.x, o.y, o.z, d0.x, d0.y, d0.z, 0.0};
  double sarc = 0.0, gam = 1.0;
  int bounce = 0, prev = -1;
  for (int iter = 0;; ++iter) {
    if (iter >= 200000) { atomicOr(A.err, kErrLoop); return; }
    if (!(y[6] < A.T_stop)) break;
    double yn[7];
    rk4_field(A, y, A.fld_h, yn);
    const D3 pos = d3(y[0], y[1], y[2]);
    const D3 chv = d3(yn[0] - y[0], yn[1] - y[1], yn[2] - y[2]);
    const double len2 = chv.x * chv.x + chv.y * chv.y + chv.z * chv.z;
    if (!(len2 > 0.0)) break;
    const double il = drsqrt_nr(len2), len = len2 * il;
    const D3 dc = d3(chv.x * il, chv.y * il, chv.z * il);
    Hit hq = closest_hit(A.sc, pos, dc, kEpsHit, len, prev >= 0 ? prev : -1, A.err);
    double ts = INFINITY;
    if (A.has_surface && prev != -2 && dc.z != 0.0) {
      const double t = (A.surface_z - pos.z) / dc.z;
      if (t > kEpsHit && t <= len) ts = t;
    }
    if (hq.prim < 0 && ts == INFINITY) {
#pragma unroll
      for (int i = 0; i < 7; ++i) y[i] = yn[i];
      sarc += A.fld_h;
      prev = -1;
      continue;
    }
    const bool surf = ts < hq.t;
    const double thit = surf ? ts : hq.t;
    const double f = thit * il;
    const double T_hit = y[6] + f * (yn[6] - y[6]), s_hit = sarc + f * A.fld_h;
    if (!(T_hit <= A.T_stop)) break;
    D3 n;
    if (surf) {
      if (bounce >= A.max_bounces) break;
      n = d3(0.0, 0.0, 1.0);
      gam *= A.r_surface;
    } else {
      const float kinc = kinc32(A.sc, hq.leaf, dc);
      const float amp = lambert(A, (float)gam, A.sc.tri_mu[hq.leaf], kinc, (float)dOmega, (float)s_hit);
      emit(A, ping, 2.0 * T_hit, amp, speckle(A, ray, sub, bounce), (float)us.y, (float)us.z, hq.prim,
           keybase | (uint32_t)bounce);
      if (!((A.sc.tri_flags[hq.leaf] & 1) && bounce < A.max_bounces)) break;
      n = tri_normal64(A.sc, hq.leaf);
      gam *= A.r_seabed;
    }
    double tg[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) tg[k] = (1.0 - f) * y[3 + k] + f * yn[3 + k];
    const double tn = sqrt(tg[0] * tg[0] + tg[1] * tg[1] + tg[2] * tg[2]);
    D3 t = d3(tg[0] / tn, tg[1] / tn, tg[2] / tn);
    const double k = 2.0 * (t.x * n.x + t.y * n.y + t.z * n.z);
    t = d3(t.x - k * n.x, t.y - k * n.y, t.z - k * n.z);
    y[0] = pos.x + thit * dc.x;
    y[1] = pos.y + thit * dc.y;
    y[2] = pos.z + thit * dc.z;
    y[3] = t.x;
    y[4] = t.y;
    y[5] = t.z;
    y[6] = T_hit;
    sarc = s_hit;
    bounce++;
    prev = surf ? -2 : hq.prim;
  }
}

__device__ void route_curved(const TraceArgs& A, int ping, D3 o, D3 d0, D3 us, uint32_t ray, uint32_t sub,
                             double dOmega, uint32_t keybase) {
  D3 pos = o;
  double ex, ey, th;
  dir_split(d0, ex, ey, th);
  double xi = cos(th) / ssp_c(A, pos.z);
  double T = 0.0, sarc = 0.0, gam = 1.0;
  int bounce = 0, prev = -1;
  for (int iter = 0;; ++iter) {
    if (iter >= 100000) { atomicOr(A.err, kErrLoop); return; }
    if (!(T < A.T_stop)) break;
    double h = arc_step(A, xi);
    Arc ar = arc_advance(A, pos.z, th, xi, h);
    D3 nxt = d3(pos.x + ar.dh * ex, pos.y + ar.dh * ey, pos.z + ar.dz);
    D3 chv = d3(nxt.x - pos.x, nxt.y - pos.y, nxt.z - pos.z);
    double len = sqrt(chv.x * chv.x + chv.y * chv.y + chv.z * chv.z);
    D3 dc = d3(chv.x / len, chv.y / len, chv.z / len);
    Hit hq = closest_hit(A.sc, pos, dc, kEpsHit, len, prev >= 0 ? prev : -1, A.err);
    double ts = INFINITY;
    if (A.has_surface && prev != -2 && dc.z != 0.0) {
      double t = (A.surface_z - pos.z) / dc.z;
      if (t > kEpsHit && t <= len) ts = t;
    }
    if (hq.prim < 0 && ts == INFINITY) {
      pos = nxt;
      th = ar.theta;
      T += ar.dt;
      sarc += h;
      prev = -1;
      continue;
    }
    bool surf = ts < hq.t;
    double thit = surf ? ts : hq.t;
    double f = thit / len;
    double T_hit = T + f * ar.dt, s_hit = sarc + f * h;
    if (!(T_hit <= A.T_stop)) break;
    D3 hp = d3(pos.x + thit * dc.x, pos.y + thit * dc.y, pos.z + thit * dc.z);
    D3 n;
    if (surf) {
      if (bounce >= A.max_bounces) break;
      n = d3(0.0, 0.0, 1.0);
      gam *= A.r_surface;
    } else {
      const float kinc = kinc32(A.sc, hq.leaf, dc);
      const float amp = lambert(A, (float)gam, A.sc.tri_mu[hq.leaf], kinc, (float)dOmega, (float)s_hit);
      emit(A, ping, 2.0 * T_hit, amp, speckle(A, ray, sub, bounce), (float)us.y, (float)us.z, hq.prim,
           keybase | (uint32_t)bounce);
      if (!((A.sc.tri_flags[hq.leaf] & 1) && bounce < A.max_bounces)) break;
      n = tri_normal64(A.sc, hq.leaf);  // FP64 only where the route continues
      gam *= A.r_seabed;
    }
    double thh = th - xi * A.ssp_g * (f * h);
    D3 tg = d3(cos(thh) * ex, cos(thh) * ey, sin(thh));
    double k = 2.0 * (tg.x * n.x + tg.y * n.y + tg.z * n.z);
    tg = d3(tg.x - k * n.x, tg.y - k * n.y, tg.z - k * n.z);
    dir_split(tg, ex, ey, th);
    pos = hp;
    xi = cos(th) / ssp_c(A, pos.z);
    T = T_hit;
    sarc = s_hit;
    bounce++;
    prev = surf ? -2 : hq.prim;
  }
}

// Cross-term multipath of a mesh hit reached after one or more reflections (Sec. II.B
// multi-bounce paths with differing outgoing and returning legs): out along the route
// and straight back to the array, and the reciprocal path, both with delay
// (L + L_d) / c and amplitude Gamma sqrt(mu cos(k_d) dOmega) / L_d exp(-alpha (L + L_d))
// (bistatic Lambertian scattering over the route's footprint; Gamma the route's one-way
// reflection product). The straight leg must reach the facet from the side the route
// arrives on and pass no other triangle closer than L_d - kCrossClear. Its geometry and
// shadow test run in FP64 from the pose; the delay adds L_d to the route's FP32-pair
// length. One speckle phase serves both paths (reciprocity), keyed apart from the
// route's own (third hash word 9 + bounce). Kept out of line: it runs for a few percent
// of hits, and inlined its FP64 leg and second traversal crowd the instruction cache of
// the route loop (ray casting with cross terms 0.139-0.142 -> 0.137 ms on C2).
constexpr double kCrossClear = 1e-4;
__device__ __noinline__ void emit_cross(const TraceArgs& A, int ping, const DevPose& P, const DF3& xh, F2 L, const DF3& dir,
                           float gam, int leaf, int prim, float dOmega, float uy, float uz, uint32_t ray,
                           uint32_t sub_i, int bounce, uint32_t keybase) {
  const D3 X = to_d3(xh);
  const D3 v = d3(X.x - P.t[0], X.y - P.t[1], X.z - P.t[2]);
  const double Ld = sqrt(dot(v, v));
  if (!(Ld > kCrossClear)) return;
  const F2 tau = (L + f2_of(Ld)) * (f2(A.two_inv_c0_df) * f2(0.5f));
  if (!(to_d(tau) <= 2.0 * A.T_stop)) return;
  const double4_32a pl = load_plane(A.sc, leaf);
  const D3 n = d3(pl.x, pl.y, pl.z);
  const double vn = dot(v, n);
  if (!(dot(to_d3(dir), n) * vn > 0.0)) return;
  const D3 ud = d3(v.x / Ld, v.y / Ld, v.z / Ld);
  const D3 o = d3(P.t[0], P.t[1], P.t[2]);
  const Hit sh = closest_hit<D3, double, true>(A.sc, o, ud, kEpsHit, Ld - kCrossClear, prim, A.err);
  if (sh.prim >= 0) return;
  const float kd = (float)(fabs(vn) / Ld) * __ldg(&A.sc.tri_inv_n[leaf]);
  const float amp = gam * sqrtf(A.sc.tri_mu[leaf] * kd * dOmega) / (float)Ld * expf(-A.alpha32 * (L.hi + (float)Ld));
  const float psi = speckle32(A, ray, sub_i, 8u + (uint32_t)bounce);
  const D3 u = rot_t(P.R, ud);
  const uint32_t key = keybase | (uint32_t)bounce;
  emit_df(A, ping, tau, amp, psi, (float)u.y, (float)u.z, prim, key | 0x40000000u);
  emit_df(A, ping, tau, amp, psi, uy, uz, prim, key | 0x20000000u);
}

template <bool CROSS>
__device__ void route_straight(const TraceArgs& A, int ping, const DevPose& P, DF3 o, const float* o32, DF3 d0,
                               float uy, float uz, uint32_t ray, uint32_t sub, float dOmega, uint32_t keybase) {
  // kEpsHit as an FP32 pair (folded at compile time)
  const F2 eps = F2{(float)kEpsHit, (float)(kEpsHit - (double)(float)kEpsHit)};
  DF3 pos = o, dir = d0;
  F2 L = f2(0.f);
  float gam = 1.0f;
  int bounce = 0, prev = -1;
  for (int iter = 0; iter < 8; ++iter) {
    const F2 tlim = f2(A.L_stop_df) - L;
    if (!(tlim.hi > 0.f)) break;
    HitT<F2> hq = closest_hit(A.sc, pos, dir, eps, tlim, prev, A.err, iter == 0 ? o32 : nullptr);
    F2 ts = F2{INFINITY, 0.f};
    // from the origin, an FP32 look first: the plane clearly behind or clearly out of
    // reach skips the exact test
    bool surf_maybe = A.has_surface && prev != -2 && dir.z.hi != 0.f;
    if (surf_maybe && iter == 0) {
      const float num32 = A.surface_z32 - o32[2], dz32 = dir.z.hi;  // tlim = L_stop at the origin
      const bool clear = fabsf(num32) > 1e-3f && fabsf(dz32) > 1e-5f;
      if (clear && (num32 * dz32 < 0.f || fabsf(num32) > A.L_stop32 * fabsf(dz32) * 1.001f + 1e-3f)) surf_maybe = false;
    }
    if (surf_maybe) {
      // divide only when the plane lies ahead within reach (a loose FP32 bound; the
      // exact test follows)
      const F2 num = f2(A.surface_z_df) - pos.z;
      if (num.hi * dir.z.hi > 0.f && fabsf(num.hi) <= tlim.hi * fabsf(dir.z.hi) * (1.0f + 1e-5f)) {
        const F2 t = num / dir.z;
        if (eps < t && !(tlim < t)) ts = t;
      }
    }
    if (hq.prim < 0 && ts.hi == INFINITY) break;
    if (ts < hq.t) {
      if (bounce >= A.max_bounces) break;
      pos = axpy(pos, ts, dir);
      L = L + ts;
      dir.z = -dir.z;
      gam *= (float)A.r_surface;
      bounce++;
      prev = -2;
      continue;
    }
    L = L + hq.t;
    const float kinc = kinc32(A.sc, hq.leaf, dir);
    const float amp = lambert(A, gam, A.sc.tri_mu[hq.leaf], kinc, dOmega, L.hi);
    emit_df(A, ping, L * f2(A.two_inv_c0_df), amp, speckle32(A, ray, sub, bounce), uy, uz, hq.prim,
            keybase | (uint32_t)bounce);
    if (CROSS && bounce > 0)
      emit_cross(A, ping, P, axpy(pos, hq.t, dir), L, dir, gam, hq.leaf, hq.prim, dOmega, uy, uz, ray, sub, bounce,
                 keybase);
    if ((A.sc.tri_flags[hq.leaf] & 1) && bounce < A.max_bounces) {
      pos = axpy(pos, hq.t, dir);
      // specular reflection off the triangle's plane: d - 2 (d . n) / (n . n) n
      F2 w;
      const DF3 n = plane_n_df(A.sc, hq.leaf, w);
      const F2 k = (dot(dir, n) + dot(dir, n)) / dot(n, n);
      dir = DF3{dir.x - k * n.x, dir.y - k * n.y, dir.z - k * n.z};
      gam *= (float)A.r_seabed;
      bounce++;
      prev = hq.prim;
      continue;
    }
    break;
  }
}

// The straight route of route_straight<false> with the warp-cooperative traversal: all
// 32 lanes step through the route's segments together (a lane whose route has ended, or
// that has no sub-ray, rides along with live = false), so every segment's closest-hit
// query is one warp-wide walk. Per lane the route, its hits and their order are those of
// route_straight.
__device__ void route_straight_warp(const TraceArgs& A, int ping, const DevPose& P, DF3 o, const float* o32, DF3 d0,
                                    float uy, float uz, uint32_t ray, uint32_t sub, float dOmega, uint32_t keybase,
                                    bool live, int* wstack) {
  const F2 eps = F2{(float)kEpsHit, (float)(kEpsHit - (double)(float)kEpsHit)};
  DF3 pos = o, dir = d0;
  F2 L = f2(0.f);
  float gam = 1.0f;
  int bounce = 0, prev = -1;
  for (int iter = 0; iter < 8; ++iter) {
    const F2 tlim = f2(A.L_stop_df) - L;
    if (!(tlim.hi > 0.f)) live = false;
    if (!__any_sync(0xffffffffu, live)) break;
    HitT<F2> hq = closest_hit_warp(A.sc, pos, dir, eps, tlim, prev, A.err, live, wstack, iter == 0 ? o32 : nullptr);
    if (!live) continue;
    F2 ts = F2{INFINITY, 0.f};
    if (A.has_surface && prev != -2 && dir.z.hi != 0.f) {
      const F2 num = f2(A.surface_z_df) - pos.z;
      if (num.hi * dir.z.hi > 0.f && fabsf(num.hi) <= tlim.hi * fabsf(dir.z.hi) * (1.0f + 1e-5f)) {
        const F2 t = num / dir.z;
        if (eps < t && !(tlim < t)) ts = t;
      }
    }
    if (hq.prim < 0 && ts.hi == INFINITY) { live = false; continue; }
    if (ts < hq.t) {
      if (bounce >= A.max_bounces) { live = false; continue; }
      pos = axpy(pos, ts, dir);
      L = L + ts;
      dir.z = -dir.z;
      gam *= (float)A.r_surface;
      bounce++;
      prev = -2;
      continue;
    }
    L = L + hq.t;
    const float kinc = kinc32(A.sc, hq.leaf, dir);
    const float amp = lambert(A, gam, A.sc.tri_mu[hq.leaf], kinc, dOmega, L.hi);
    emit_df(A, ping, L * f2(A.two_inv_c0_df), amp, speckle32(A, ray, sub, bounce), uy, uz, hq.prim,
            keybase | (uint32_t)bounce);
    if ((A.sc.tri_flags[hq.leaf] & 1) && bounce < A.max_bounces) {
      pos = axpy(pos, hq.t, dir);
      F2 w;
      const DF3 n = plane_n_df(A.sc, hq.leaf, w);
      const F2 k = (dot(dir, n) + dot(dir, n)) / dot(n, n);
      dir = DF3{dir.x - k * n.x, dir.y - k * n.y, dir.z - k * n.z};
      gam *= (float)A.r_seabed;
      bounce++;
      prev = hq.prim;
      continue;
    }
    live = false;
  }
}

// Straight rays with the warp-cooperative traversal: each warp takes 32 consecutive
// sub-rays (neighbouring azimuth cells and their sub-rays: nearly parallel rays).
__global__ void __launch_bounds__(128) k_trace_warp(TraceArgs A) {
  __shared__ int wstack[4][kMaxStack];
  pdl_wait();
  const int64_t total = (int64_t)A.n_pings * A.n_subrays;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + w) * 32; base < total; base += warps * 32) {
    const int64_t gid = base + lane;
    const bool live = gid < total;
    const int64_t g = live ? gid : total - 1;
    int ping = (int)(g / A.n_subrays);
    int sr = (int)(g % A.n_subrays);
    uint32_t ray = (uint32_t)(sr / A.n_sub), sub = (uint32_t)(sr % A.n_sub);
    int row = (int)(ray / A.n_ray_az);
    const DevPose& P = A.poses[ping];
    const float dOmega = A.row_domega[row];
    const uint32_t keybase = ((uint32_t)sr) << 2;
    const float* uh = A.ray_dirs32 + 3 * sr;
    const float* ul = A.ray_dirs_lo + 3 * sr;
    const F2 u[3] = {F2{uh[0], ul[0]}, F2{uh[1], ul[1]}, F2{uh[2], ul[2]}};
    F2 dw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      dw[i] = F2{P.R32[3 * i], P.R_lo[3 * i]} * u[0] + F2{P.R32[3 * i + 1], P.R_lo[3 * i + 1]} * u[1] +
              F2{P.R32[3 * i + 2], P.R_lo[3 * i + 2]} * u[2];
    const DF3 o = DF3{F2{P.t32[0], P.t_lo[0]}, F2{P.t32[1], P.t_lo[1]}, F2{P.t32[2], P.t_lo[2]}};
    route_straight_warp(A, ping, P, o, P.t32, DF3{dw[0], dw[1], dw[2]}, uh[1], uh[2], ray, sub, dOmega, keybase, live,
                        wstack[w]);
  }
}

// Traversal is latency-bound (dependent node loads), so residency pays: the straight-ray
// kernel runs seven CTAs of 128 threads per SM (72 registers, an 80-byte spill; measured
// on C2 with one copy of the leaf test in the loop: 5 CTAs 0.098 ms, 6 0.092, 7 0.088, 8
// 0.093), the curved one four. The cross-term variant is a separate instantiation, so
// that its extra live state does not
// cost the default kernel registers.
#ifndef SONAR_TRACE_CTAS
#define SONAR_TRACE_CTAS 7  // resident CTAs per SM of the straight-ray kernel
#endif
template <bool CURVED, bool CROSS>
__global__ void __launch_bounds__(128, CURVED ? 4 : SONAR_TRACE_CTAS) k_trace(TraceArgs A) {
  pdl_wait();
  const int64_t total = (int64_t)A.n_pings * A.n_subrays;
  for (int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gid < total; gid += (int64_t)gridDim.x * blockDim.x) {
    int ping = (int)(gid / A.n_subrays);
    int sr = (int)(gid % A.n_subrays);
    uint32_t ray = (uint32_t)(sr / A.n_sub), sub = (uint32_t)(sr % A.n_sub);
    int row = (int)(ray / A.n_ray_az);
    const DevPose& P = A.poses[ping];
    const float dOmega = A.row_domega[row];
    const uint32_t keybase = ((uint32_t)sr) << 2;
    if (CURVED) {
      const D3 us = d3(A.ray_dirs[3 * sr], A.ray_dirs[3 * sr + 1], A.ray_dirs[3 * sr + 2]);
      const D3 dw = rot(P.R, us);
      const D3 o = d3(P.t[0], P.t[1], P.t[2]);
      if (A.fld_nx > 0) route_field(A, ping, o, dw, us, ray, sub, dOmega, keybase);
      else route_curved(A, ping, o, dw, us, ray, sub, dOmega, keybase);
    } else {
      // world direction R us and origin t as FP32 pairs
      const float* uh = A.ray_dirs32 + 3 * sr;
      const float* ul = A.ray_dirs_lo + 3 * sr;
      const F2 u[3] = {F2{uh[0], ul[0]}, F2{uh[1], ul[1]}, F2{uh[2], ul[2]}};
      F2 dw[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        dw[i] = F2{P.R32[3 * i], P.R_lo[3 * i]} * u[0] + F2{P.R32[3 * i + 1], P.R_lo[3 * i + 1]} * u[1] +
                F2{P.R32[3 * i + 2], P.R_lo[3 * i + 2]} * u[2];
      const DF3 o = DF3{F2{P.t32[0], P.t_lo[0]}, F2{P.t32[1], P.t_lo[1]}, F2{P.t32[2], P.t_lo[2]}};
      route_straight<CROSS>(A, ping, P, o, P.t32, DF3{dw[0], dw[1], dw[2]}, uh[1], uh[2], ray, sub, dOmega, keybase);
    }
  }
}

// ----------------------------------------------------------------- point scatterers
__device__ bool leg_clear(const TraceArgs& A, D3 a, D3 b) {
  D3 d = sub(b, a);
  double len = sqrt(dot(d, d));
  if (len <= 2e-6) return true;
  d = d3(d.x / len, d.y / len, d.z / len);
  Hit h = closest_hit<D3, double, true>(A.sc, a, d, 1e-6, len - 1e-6, -1, A.err);
  return h.prim < 0;
}

__device__ D3 mirror(const double4_32a pl, D3 x) {
  double k = 2.0 * (pl.x * x.x + pl.y * x.y + pl.z * x.z - pl.w);
  return d3(x.x - k * pl.x, x.y - k * pl.y, x.z - k * pl.z);
}

__device__ double4_32a plane_of(const TraceArgs& A, int idx, double& gam) {
  if (A.has_surface) {
    if (idx == 0) { gam = A.r_surface; return make_double4_32a(0.0, 0.0, 1.0, A.surface_z); }
    idx -= 1;
  }
  gam = A.r_seabed;
  return A.sc.planes[idx];
}

// Monostatic image-source eigen-routes of a point scatterer (isovelocity), or its
// direct eigen-arc in a linear profile. Routes are plane sequences without immediate
// repeats, enumerated by length then lexicographically.
__global__ void k_points(TraceArgs A) {
  pdl_wait();
  int64_t total = (int64_t)A.n_pings * A.sc.n_points * A.n_routes;
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= total) return;
  int route = (int)(gid % A.n_routes);
  int ip = (int)((gid / A.n_routes) % A.sc.n_points);
  int ping = (int)(gid / ((int64_t)A.n_routes * A.sc.n_points));
  const DevPose& P = A.poses[ping];
  float4 xp = A.sc.points[ip];
  D3 x = d3(xp.x, xp.y, xp.z);
  D3 o = d3(P.t[0], P.t[1], P.t[2]);
  double sigma = xp.w;
  uint32_t key = 0x80000000u | ((uint32_t)ip << 8) | (uint32_t)route;
  if (A.cross) A.pt_route[gid] = PtRoute{0.0, 0.0, 0.f, 0.f, 0, 0};  // invalid until it passes
  if (A.curved) {
    if (route != 0) return;
    double dx = x.x - o.x, dy = x.y - o.y;
    double D = sqrt(dx * dx + dy * dy);
    double co = ssp_c(A, o.z), cx = ssp_c(A, x.z);
    double g = A.ssp_g;
    D3 dw;
    double T, sarc;
    if (D == 0.0) {
      double dzz = x.z - o.z;
      dw = d3(0.0, 0.0, dzz > 0 ? 1.0 : -1.0);
      T = log(cx / co) / (g * dw.z);
      sarc = fabs(dzz);
    } else {
      double ex = dx / D, ey = dy / D;
      double a = co / g, b = cx / g;
      double hc = (D * D + b * b - a * a) / (2 * D);
      double Rr = sqrt(hc * hc + a * a);
      double sg = g > 0 ? 1.0 : -1.0;
      double th0 = atan2(sg * hc, sg * a), th1 = atan2(sg * (hc - D), sg * b);
      dw = d3(cos(th0) * ex, cos(th0) * ey, sin(th0));
      double s0 = sin(th0), s1 = sin(th1);
      double X = (s0 - s1) / (1 - s0 * s1);
      T = atanh(X) / g;
      double ang = atan2(fabs(-hc * b - a * (D - hc)), -hc * (D - hc) + a * b);
      sarc = Rr * ang;
    }
    if (!(T <= A.T_stop)) return;
    D3 pos = o;
    double ex, ey, th;
    dir_split(dw, ex, ey, th);
    double xi = cos(th) / ssp_c(A, pos.z);
    double left = sarc;
    for (int it = 0; left > 0 && it < 100000; ++it) {
      double h = fmin(arc_step(A, xi), left);
      Arc ar = arc_advance(A, pos.z, th, xi, h);
      D3 nxt = d3(pos.x + ar.dh * ex, pos.y + ar.dh * ey, pos.z + ar.dz);
      if (left - h <= 0) nxt = x;
      if (!leg_clear(A, pos, nxt)) return;
      pos = nxt;
      th = ar.theta;
      left -= h;
    }
    double amp = sigma / (sarc * sarc) * exp(-2.0 * A.alpha * sarc);
    const D3 u = rot_t(P.R, dw);
    emit(A, ping, 2.0 * T, (float)amp, 0.0, (float)u.y, (float)u.z, -1, key);
    return;
  }
  int np = (A.has_surface ? 1 : 0) + A.sc.n_planes;
  // decode the route index into a plane sequence
  int len = 0;
  int64_t r = route, count = 1;
  while (r >= count) {
    r -= count;
    ++len;
    count = np;
    for (int k = 1; k < len; ++k) count *= (np - 1);
    if (np == 0 || len > A.max_bounces) return;
  }
  int seq[4];
  int64_t div = 1;
  for (int k = 1; k < len; ++k) div *= (np - 1);
  for (int k = 0; k < len; ++k) {
    int64_t digit = r / div;
    r %= div;
    if (k + 1 < len) div /= (np - 1);
    seq[k] = k == 0 ? (int)digit : ((int)digit < seq[k - 1] ? (int)digit : (int)digit + 1);
  }
  D3 img = x;
  double gam = 1.0;
  for (int k = len - 1; k >= 0; --k) {
    double gk;
    img = mirror(plane_of(A, seq[k], gk), img);
    gam *= gk;
  }
  D3 dv = sub(img, o);
  double L = sqrt(dot(dv, dv));
  if (!(L > 0) || !(L / A.ssp_c0 <= A.T_stop)) return;
  D3 a = o, tgt = img;
  for (int k = 0; k < len; ++k) {
    double gk;
    double4_32a pl = plane_of(A, seq[k], gk);
    double dA = pl.x * a.x + pl.y * a.y + pl.z * a.z - pl.w;
    double dT = pl.x * tgt.x + pl.y * tgt.y + pl.z * tgt.z - pl.w;
    if (!(dA * dT < 0)) return;
    double f = dA / (dA - dT);
    D3 sp = d3(a.x + f * (tgt.x - a.x), a.y + f * (tgt.y - a.y), a.z + f * (tgt.z - a.z));
    if (!leg_clear(A, a, sp)) return;
    tgt = mirror(pl, tgt);
    a = sp;
  }
  if (!leg_clear(A, a, x)) return;
  double amp = sigma * gam * gam / (L * L) * exp(-2.0 * A.alpha * L);
  D3 dw = d3(dv.x / L, dv.y / L, dv.z / L);
  const D3 u = rot_t(P.R, dw);
  emit(A, ping, 2.0 * L / A.ssp_c0, (float)amp, 0.0, (float)u.y, (float)u.z, -1, key);
  if (A.cross) A.pt_route[gid] = PtRoute{L, gam, (float)u.y, (float)u.z, len, 0};
}

// Cross pairs of a point scatterer's routes: out along route i, back along route j != i,
// delay (L_i + L_j) / c, amplitude sigma Gamma_i Gamma_j / (L_i L_j) exp(-alpha
// (L_i + L_j)), arriving along route j; no speckle. Reads the routes k_points recorded.
__global__ void k_point_pairs(TraceArgs A) {
  pdl_wait();
  const int nr = A.n_routes;
  const int64_t total = (int64_t)A.n_pings * A.sc.n_points * nr * nr;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= total) return;
  const int j = (int)(gid % nr), i = (int)((gid / nr) % nr);
  const int64_t pt = gid / ((int64_t)nr * nr);  // ping * n_points + point
  if (i == j) return;
  const PtRoute a = A.pt_route[pt * nr + i], b = A.pt_route[pt * nr + j];
  if (!(a.L > 0.0) || !(b.L > 0.0)) return;
  const int ip = (int)(pt % A.sc.n_points), ping = (int)(pt / A.sc.n_points);
  const double Ls = a.L + b.L;
  const double amp = (double)A.sc.points[ip].w * a.gam * b.gam / (a.L * b.L) * exp(-A.alpha * Ls);
  const uint32_t key = 0xC0000000u | ((uint32_t)ip << 16) | ((uint32_t)i << 8) | (uint32_t)j;
  emit(A, ping, Ls / A.ssp_c0, (float)amp, 0.0, b.uy, b.uz, -1, key);
}

// Water-column reverberation (Sec. II.B volumetric backscatter paths): scatterer i of
// the world-frame box sits at lo + (hi - lo) u, u the first three 24-bit fractions of
// pcg4d(i mod 2^32, i div 2^32, 0x564F4C, seed) (products and sums rounded separately);
// it echoes on its direct route when the leg is clear: amplitude sigma / L^2
// exp(-2 alpha L), delay 2 L / c, no speckle phase. One thread per (ping, scatterer),
// taken in the Morton order of the positions when the host has sorted them, so that the
// shadow legs of a warp run to neighbouring points and traverse the same nodes.
__global__ void k_volume(TraceArgs A) {
  pdl_wait();
  const int64_t total = (int64_t)A.n_pings * A.vol_n;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= total) return;
  const int64_t i = A.vol_order ? (int64_t)A.vol_order[gid % A.vol_n] : gid % A.vol_n;
  const int ping = (int)(gid / A.vol_n);
  uint32_t h[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0x564F4Cu, A.seed32};
  pcg4d(h[0], h[1], h[2], h[3]);
  // geometry and delay in FP32 pairs, as on the straight-ray path (FP64 issues at ~2
  // operations per clock per SM on this part): the position lo + (hi - lo) u (u, a
  // 24-bit fraction, is exact in FP32), the leg, its length and direction, and the
  // shadow query's near-tie triangle tests
  const DevPose& P = A.poses[ping];
  const DF3 o = DF3{F2{P.t32[0], P.t_lo[0]}, F2{P.t32[1], P.t_lo[1]}, F2{P.t32[2], P.t_lo[2]}};
  F2 dvk[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const F2 u = f2((float)(h[k] >> 8) * (1.0f / 16777216.0f));
    dvk[k] = f2(A.vol_lo_df[k]) + f2(A.vol_span_df[k]) * u;
  }
  const DF3 dv = DF3{dvk[0] - o.x, dvk[1] - o.y, dvk[2] - o.z};
  const F2 L = sqrt_df(dot(dv, dv));
  if (!(L.hi > 0.f) || f2(A.L_stop_df) < L) return;
  const F2 il = f2(1.f) / L;
  const DF3 d = DF3{dv.x * il, dv.y * il, dv.z * il};
  if (L.hi > 2e-6f) {
    const F2 eps = F2{1e-6f, (float)(1e-6 - (double)1e-6f)};
    if (closest_hit<DF3, F2, true>(A.sc, o, d, eps, L - eps, -1, A.err, P.t32).prim >= 0) return;
  }
  const float amp = (float)A.vol_sigma / (L.hi * L.hi) * expf(-2.0f * A.alpha32 * L.hi);
  const float uy = P.R32[1] * d.x.hi + P.R32[4] * d.y.hi + P.R32[7] * d.z.hi;  // (R^T d).y
  const float uz = P.R32[2] * d.x.hi + P.R32[5] * d.y.hi + P.R32[8] * d.z.hi;  // (R^T d).z
  emit_df(A, ping, L * f2(A.two_inv_c0_df), amp, 0.f, uy, uz, -1, 0xA0000000u | (uint32_t)i);
}

// Sonar-frame sub-ray directions (Sec. III Eq. 2-3 grid, cell-centred) with hashed
// jitter inside 2x2 quarter cells, and the sub-ray solid angle per elevation row.
// Geometric rendering of the learned surrogate: one ray per beam along the beam centre,
// routed by the same straight-ray rules as route_straight (mirror facets and the sea
// surface reflect, at most max_bounces, up to the one-way length limit). Records the
// first two scatter (triangle) hits of the route: one-way length L, incidence cosine,
// facet reflectivity and the route's one-way reflection product, zeros where absent.
// feat: [n_pings][n_beam_el * n_beam_az][8].
__global__ void __launch_bounds__(128) k_render(TraceArgs A, int nba, int nbe, double hfov, double vfov, float* feat) {
  pdl_wait();
  const int nb = nba * nbe;
  const int64_t total = (int64_t)A.n_pings * nb;
  const F2 eps = F2{(float)kEpsHit, (float)(kEpsHit - (double)(float)kEpsHit)};
  for (int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gid < total; gid += (int64_t)gridDim.x * blockDim.x) {
    const int ping = (int)(gid / nb), b = (int)(gid % nb);
    const int i = b % nba, j = b / nba;
    const double az = -hfov / 2 + (i + 0.5) * hfov / nba;
    const double el = -vfov / 2 + (j + 0.5) * vfov / nbe;
    const double us[3] = {cos(el) * cos(az), cos(el) * sin(az), sin(el)};
    F2 u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = f2_of(us[k]);
    const DevPose& P = A.poses[ping];
    F2 dw[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      dw[k] = F2{P.R32[3 * k], P.R_lo[3 * k]} * u[0] + F2{P.R32[3 * k + 1], P.R_lo[3 * k + 1]} * u[1] +
              F2{P.R32[3 * k + 2], P.R_lo[3 * k + 2]} * u[2];
    DF3 pos = DF3{F2{P.t32[0], P.t_lo[0]}, F2{P.t32[1], P.t_lo[1]}, F2{P.t32[2], P.t_lo[2]}};
    DF3 dir = DF3{dw[0], dw[1], dw[2]};
    float out[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    F2 L = f2(0.f);
    float gam = 1.0f;
    int bounce = 0, prev = -1, n_hit = 0;
    for (int iter = 0; iter < 8 && n_hit < 2; ++iter) {
      const F2 tlim = f2(A.L_stop_df) - L;
      if (!(tlim.hi > 0.f)) break;
      HitT<F2> hq = closest_hit(A.sc, pos, dir, eps, tlim, prev, A.err, iter == 0 ? P.t32 : nullptr);
      F2 ts = F2{INFINITY, 0.f};
      if (A.has_surface && prev != -2 && dir.z.hi != 0.f) {
        const F2 num = f2(A.surface_z_df) - pos.z;
        if (num.hi * dir.z.hi > 0.f && fabsf(num.hi) <= tlim.hi * fabsf(dir.z.hi) * (1.0f + 1e-5f)) {
          const F2 t = num / dir.z;
          if (eps < t && !(tlim < t)) ts = t;
        }
      }
      if (hq.prim < 0 && ts.hi == INFINITY) break;
      if (ts < hq.t) {
        if (bounce >= A.max_bounces) break;
        pos = axpy(pos, ts, dir);
        L = L + ts;
        dir.z = -dir.z;
        gam *= (float)A.r_surface;
        bounce++;
        prev = -2;
        continue;
      }
      L = L + hq.t;
      out[4 * n_hit] = L.hi + L.lo;
      out[4 * n_hit + 1] = kinc32(A.sc, hq.leaf, dir);
      out[4 * n_hit + 2] = A.sc.tri_mu[hq.leaf];
      out[4 * n_hit + 3] = gam;
      ++n_hit;
      if ((A.sc.tri_flags[hq.leaf] & 1) && bounce < A.max_bounces) {
        pos = axpy(pos, hq.t, dir);
        F2 w;
        const DF3 n = plane_n_df(A.sc, hq.leaf, w);
        const F2 k = (dot(dir, n) + dot(dir, n)) / dot(n, n);
        dir = DF3{dir.x - k * n.x, dir.y - k * n.y, dir.z - k * n.z};
        gam *= (float)A.r_seabed;
        bounce++;
        prev = hq.prim;
        continue;
      }
      break;
    }
    float4* o4 = reinterpret_cast<float4*>(feat + gid * 8);
    o4[0] = make_float4(out[0], out[1], out[2], out[3]);
    o4[1] = make_float4(out[4], out[5], out[6], out[7]);
  }
}

__global__ void k_ray_table(double* dirs, float* dirs32, float* row_domega, int nra, int nre, int nsub, double hfov,
                            double vfov, uint32_t seed32) {
  int64_t n = (int64_t)nra * nre * nsub;
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double daz = hfov / nra, del = vfov / nre;
  if (gid < nre) {
    double el_lo = -vfov / 2 + gid * del, el_hi = el_lo + del;
    row_domega[gid] = (float)(daz * (sin(el_hi) - sin(el_lo)) / nsub);
  }
  if (gid >= n) return;
  int s = (int)(gid % nsub);
  int ray = (int)(gid / nsub);
  int i = ray % nra, j = ray / nra;
  double ox = 0.0, oy = 0.0;
  if (nsub == 4) {
    uint32_t x = (uint32_t)ray, y = (uint32_t)s, z = 0u, w = seed32;
    pcg4d(x, y, z, w);
    ox = ((s & 1) + u24(x)) / 2.0 - 0.5;
    oy = ((s >> 1) + u24(y)) / 2.0 - 0.5;
  }
  double az = -hfov / 2 + (i + 0.5 + ox) * daz;
  double el = -vfov / 2 + (j + 0.5 + oy) * del;
  dirs[3 * gid] = cos(el) * cos(az);
  dirs[3 * gid + 1] = cos(el) * sin(az);
  dirs[3 * gid + 2] = sin(el);
  for (int k = 0; k < 3; ++k) {
    const float hi = (float)dirs[3 * gid + k];
    dirs32[3 * gid + k] = hi;
    dirs32[3 * n + 3 * gid + k] = (float)(dirs[3 * gid + k] - (double)hi);
  }
}

}  // namespace

cudaError_t launch_point_pairs(const TraceArgs& a, cudaStream_t st) {
  const int64_t total = (int64_t)a.n_pings * a.sc.n_points * a.n_routes * a.n_routes;
  if (total == 0) return cudaSuccess;
  cudaError_t e = launch_pdl(k_point_pairs, dim3((unsigned)ceil_div(total, 128)), dim3(128), 0, st, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_volume(const TraceArgs& a, cudaStream_t st) {
  const int64_t total = (int64_t)a.n_pings * a.vol_n;
  if (total == 0) return cudaSuccess;
  cudaError_t e = launch_pdl(k_volume, dim3((unsigned)ceil_div(total, 128)), dim3(128), 0, st, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_ray_table(double* dirs, float* dirs32, float* row_domega, int32_t nra, int32_t nre, int32_t nsub,
                             double hfov, double vfov, uint32_t seed32, cudaStream_t st) {
  int64_t n = (int64_t)nra * nre * nsub;
  if (n < nre) n = nre;
  k_ray_table<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(dirs, dirs32, row_domega, nra, nre, nsub, hfov, vfov,
                                                          seed32);
  return cudaGetLastError();
}

cudaError_t launch_trace(const TraceArgs& a, int sm_count, cudaStream_t st) {
  int64_t total = (int64_t)a.n_pings * a.n_subrays;
  int64_t blocks = ceil_div(total, 128);
  // one sub-ray per thread: the block scheduler balances the uneven route lengths. A
  // cap of 16 blocks per SM (two grid-stride passes for 40% of the blocks on C2) left an
  // uneven tail: 0.123 ms against 0.106 ms uncapped.
  const int64_t cap = 0x7fffffffLL;  // the grid limit
  (void)sm_count;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  cudaError_t e = a.curved      ? launch_pdl(k_trace<true, false>, dim3((unsigned)blocks), dim3(128), 0, st, a)
                  : a.cross     ? launch_pdl(k_trace<false, true>, dim3((unsigned)blocks), dim3(128), 0, st, a)
                  : a.warp_walk ? launch_pdl(k_trace_warp, dim3((unsigned)blocks), dim3(128), 0, st, a)
                                : launch_pdl(k_trace<false, false>, dim3((unsigned)blocks), dim3(128), 0, st, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_render(const TraceArgs& a, int32_t nba, int32_t nbe, double hfov, double vfov, float* feat,
                          cudaStream_t st) {
  const int64_t total = (int64_t)a.n_pings * nba * nbe;
  if (total == 0) return cudaSuccess;
  k_render<<<(unsigned)ceil_div(total, 128), 128, 0, st>>>(a, nba, nbe, hfov, vfov, feat);
  return cudaGetLastError();
}

cudaError_t launch_points(const TraceArgs& a, cudaStream_t st) {
  int64_t total = (int64_t)a.n_pings * a.sc.n_points * a.n_routes;
  if (total == 0) return cudaSuccess;
  cudaError_t e = launch_pdl(k_points, dim3((unsigned)ceil_div(total, 64)), dim3(64), 0, st, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace sonar
