// Scene BVH on the device: linear BVH (Karras 2012, "Maximizing parallelism in the
// construction of BVHs, octrees and k-d trees") over triangle centroids.
// Morton codes -> bitonic sort -> hierarchy from key prefixes -> bottom-up boxes ->
// 64-byte two-child nodes, with triangles reordered into leaf order. Run once per
// scene upload; the per-ping path only reads the result. Boxes are widened so that the
// FP32 traversal never culls a triangle the FP64 decision would accept.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace sonar {
namespace {

__device__ inline float atomic_min_f(float* a, float v) {
  return v >= 0.f ? __int_as_float(atomicMin((int*)a, __float_as_int(v)))
                  : __uint_as_float(atomicMax((unsigned*)a, __float_as_uint(v)));
}
__device__ inline float atomic_max_f(float* a, float v) {
  return v >= 0.f ? __int_as_float(atomicMax((int*)a, __float_as_int(v)))
                  : __uint_as_float(atomicMin((unsigned*)a, __float_as_uint(v)));
}

__device__ inline void load_tri(const float* V, const int32_t* T, int i, float3& a, float3& b, float3& c) {
  int ia = T[3 * i], ib = T[3 * i + 1], ic = T[3 * i + 2];
  a = make_float3(V[3 * ia], V[3 * ia + 1], V[3 * ia + 2]);
  b = make_float3(V[3 * ib], V[3 * ib + 1], V[3 * ib + 2]);
  c = make_float3(V[3 * ic], V[3 * ic + 1], V[3 * ic + 2]);
}

__global__ void k_bounds(const float* V, const int32_t* T, int n, float* bb) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float3 a, b, c;
    load_tri(V, T, i, a, b, c);
    float ce[3] = {(a.x + b.x + c.x) / 3.f, (a.y + b.y + c.y) / 3.f, (a.z + b.z + c.z) / 3.f};
    for (int k = 0; k < 3; ++k) { lo[k] = fminf(lo[k], ce[k]); hi[k] = fmaxf(hi[k], ce[k]); }
  }
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < 3; ++k) { atomic_min_f(&bb[k], lo[k]); atomic_max_f(&bb[3 + k], hi[k]); }
  }
}

__device__ inline uint32_t expand10(uint32_t v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

__global__ void k_morton(const float* V, const int32_t* T, int n, int n_pow2, const float* bb,
                         unsigned long long* keys) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pow2) return;
  if (i >= n) { keys[i] = ~0ull; return; }
  float3 a, b, c;
  load_tri(V, T, i, a, b, c);
  float ce[3] = {(a.x + b.x + c.x) / 3.f, (a.y + b.y + c.y) / 3.f, (a.z + b.z + c.z) / 3.f};
  uint32_t q[3];
  for (int k = 0; k < 3; ++k) {
    float ext = bb[3 + k] - bb[k];
    float f = ext > 0.f ? (ce[k] - bb[k]) / ext : 0.5f;
    q[k] = (uint32_t)fminf(fmaxf(f * 1024.f, 0.f), 1023.f);
  }
  uint32_t m = (expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]);
  keys[i] = ((unsigned long long)m << 32) | (unsigned)i;
}

__global__ void k_bitonic(unsigned long long* keys, int n_pow2, int k, int j) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pow2) return;
  int l = i ^ j;
  if (l <= i) return;
  unsigned long long a = keys[i], b = keys[l];
  bool up = (i & k) == 0;
  if ((a > b) == up) { keys[i] = b; keys[l] = a; }
}

__device__ inline int delta(const unsigned long long* keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  return __clzll(keys[i] ^ keys[j]);
}

// Karras 2012, Fig. 4: node i covers a key range found from the common prefix with
// its neighbours; the split is where the prefix length first drops.
__global__ void k_hierarchy(const unsigned long long* keys, int n, int2* child, int* par_int, int* par_leaf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(keys, n, i, i - d);
  int lmax = 2;
  while (delta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
  int l = 0;
  for (int t = lmax / 2; t >= 1; t /= 2)
    if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = delta(keys, n, i, j);
  int s = 0, div = 2, t;
  do {
    t = (l + div - 1) / div;
    if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    div *= 2;
  } while (t > 1);
  int g = i + s * d + min(d, 0);
  int left = (min(i, j) == g) ? ~g : g;
  int right = (max(i, j) == g + 1) ? ~(g + 1) : g + 1;
  child[i] = make_int2(left, right);
  if (left < 0) par_leaf[~left] = i; else par_int[left] = i;
  if (right < 0) par_leaf[~right] = i; else par_int[right] = i;
  if (i == 0) par_int[0] = -1;
}

__global__ void k_leaves(const float* V, const int32_t* T, const float* mu, const uint8_t* fl,
                         const unsigned long long* keys, int n, float4* lbox_lo, float4* lbox_hi,
                         float4* tri32, float* triv, int32_t* tri_prim, float* tri_mu, uint8_t* tri_flags,
                         double4_32a* tri_plane, float* tri_inv_n) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int prim = (int)(keys[k] & 0xffffffffu);
  float3 a, b, c;
  load_tri(V, T, prim, a, b, c);
  lbox_lo[k] = make_float4(fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y)), fminf(a.z, fminf(b.z, c.z)), 0.f);
  lbox_hi[k] = make_float4(fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y)), fmaxf(a.z, fmaxf(b.z, c.z)), 0.f);
  tri32[3 * k] = make_float4(a.x, a.y, a.z, 0.f);
  tri32[3 * k + 1] = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, 0.f);
  tri32[3 * k + 2] = make_float4(c.x - a.x, c.y - a.y, c.z - a.z, 0.f);
  float v[9] = {a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z};
  for (int q = 0; q < 9; ++q) triv[9 * k + q] = v[q];
  tri_prim[k] = prim;
  tri_mu[k] = mu[prim];
  tri_flags[k] = fl[prim];
  // FP64 plane: float vertex differences are exact in FP64; unrounded product order
  const double e1x = __dsub_rn(b.x, a.x), e1y = __dsub_rn(b.y, a.y), e1z = __dsub_rn(b.z, a.z);
  const double e2x = __dsub_rn(c.x, a.x), e2y = __dsub_rn(c.y, a.y), e2z = __dsub_rn(c.z, a.z);
  const double nx = __dsub_rn(__dmul_rn(e1y, e2z), __dmul_rn(e1z, e2y));
  const double ny = __dsub_rn(__dmul_rn(e1z, e2x), __dmul_rn(e1x, e2z));
  const double nz = __dsub_rn(__dmul_rn(e1x, e2y), __dmul_rn(e1y, e2x));
  const double d0 = __dadd_rn(__dadd_rn(__dmul_rn(nx, (double)a.x), __dmul_rn(ny, (double)a.y)), __dmul_rn(nz, (double)a.z));
  tri_plane[k] = make_double4_32a(nx, ny, nz, d0);
  // FP32 pairs of the plane after the n FP64 planes: hi = RN(x), lo = RN(x - hi)
  float4* df = reinterpret_cast<float4*>(tri_plane + n);
  const float hx = (float)nx, hy = (float)ny, hz = (float)nz, hw = (float)d0;
  df[2 * k] = make_float4(hx, hy, hz, hw);
  df[2 * k + 1] = make_float4((float)(nx - (double)hx), (float)(ny - (double)hy), (float)(nz - (double)hz),
                              (float)(d0 - (double)hw));
  const double nn = __dadd_rn(__dadd_rn(__dmul_rn(nx, nx), __dmul_rn(ny, ny)), __dmul_rn(nz, nz));
  tri_inv_n[k] = nn > 0.0 ? (float)(1.0 / sqrt(nn)) : 0.f;
}

__global__ void k_refit(int n, const int2* child, const int* par_int, const int* par_leaf,
                        const float4* lbox_lo, const float4* lbox_hi, float4* ibox_lo, float4* ibox_hi,
                        int* flags) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int p = par_leaf[k];
  while (p >= 0) {
    __threadfence();
    if (atomicAdd(&flags[p], 1) == 0) return;
    int2 ch = child[p];
    float4 lo0, hi0, lo1, hi1;
    if (ch.x < 0) { lo0 = lbox_lo[~ch.x]; hi0 = lbox_hi[~ch.x]; }
    else { lo0 = __ldcg(&ibox_lo[ch.x]); hi0 = __ldcg(&ibox_hi[ch.x]); }
    if (ch.y < 0) { lo1 = lbox_lo[~ch.y]; hi1 = lbox_hi[~ch.y]; }
    else { lo1 = __ldcg(&ibox_lo[ch.y]); hi1 = __ldcg(&ibox_hi[ch.y]); }
    __stcg(&ibox_lo[p], make_float4(fminf(lo0.x, lo1.x), fminf(lo0.y, lo1.y), fminf(lo0.z, lo1.z), 0.f));
    __stcg(&ibox_hi[p], make_float4(fmaxf(hi0.x, hi1.x), fmaxf(hi0.y, hi1.y), fmaxf(hi0.z, hi1.z), 0.f));
    p = par_int[p];
  }
}

__device__ inline float widen_lo(float v) { return v - (1e-4f + 1e-6f * fabsf(v)); }
__device__ inline float widen_hi(float v) { return v + (1e-4f + 1e-6f * fabsf(v)); }

__global__ void k_pack(int n_int, const int2* child, const float4* lbox_lo, const float4* lbox_hi,
                       const float4* ibox_lo, const float4* ibox_hi, BvhNode* nodes) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_int) return;
  int2 ch = child[i];
  float4 L0 = ch.x < 0 ? lbox_lo[~ch.x] : ibox_lo[ch.x];
  float4 L1 = ch.x < 0 ? lbox_hi[~ch.x] : ibox_hi[ch.x];
  float4 R0, R1;
  if (ch.y == INT_MIN) {  // no right child (one-triangle scene): a point at 1e30 m
    R0 = make_float4(1e30f, 1e30f, 1e30f, 0.f);
    R1 = R0;
  } else {
    R0 = ch.y < 0 ? lbox_lo[~ch.y] : ibox_lo[ch.y];
    R1 = ch.y < 0 ? lbox_hi[~ch.y] : ibox_hi[ch.y];
  }
  BvhNode nd;
  nd.a = make_float4(widen_lo(L0.x), widen_hi(L1.x), widen_lo(L0.y), widen_hi(L1.y));
  nd.b = make_float4(widen_lo(R0.x), widen_hi(R1.x), widen_lo(R0.y), widen_hi(R1.y));
  nd.c = make_float4(widen_lo(L0.z), widen_hi(L1.z), widen_lo(R0.z), widen_hi(R1.z));
  nd.d = make_int4(ch.x, ch.y, 0, 0);
  nodes[i] = nd;
}

__global__ void k_single(int2* child) { child[0] = make_int2(~0, INT_MIN); }

}  // namespace

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return e_; } while (0)

// ----------------------------------------------------------------- binned SAH (host)
// Top-down build with the surface area heuristic over 16 centroid bins per split (Wald,
// "On fast construction of SAH-based bounding volume hierarchies", 2007), one triangle
// per leaf. It produces the same hierarchy arrays as the Morton-order build (children of
// internal node i, parents, leaf order), so the device refit and packing are shared.
// Fewer node visits per ray than the Morton order on scenes like a corrugated wall over
// a rough seabed; the build is sequential host work, once per scene.
namespace {
struct SahTri {
  float lo[3], hi[3], c[3];
};
struct Box3 {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  void grow(const float* l, const float* h) {
    for (int k = 0; k < 3; ++k) { lo[k] = fminf(lo[k], l[k]); hi[k] = fmaxf(hi[k], h[k]); }
  }
  float area() const {
    if (!(hi[0] >= lo[0])) return 0.f;
    const float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return 2.f * (dx * dy + dy * dz + dz * dx);
  }
};

// keys[k] = original id of leaf k; child[i] (>= 0: internal node, < 0: ~leaf); parents
void sah_build(const float* V, const int32_t* T, int n, std::vector<unsigned long long>& keys,
               std::vector<int2>& child, std::vector<int>& par_int, std::vector<int>& par_leaf) {
  constexpr int kBins = 16;
  std::vector<SahTri> tri(n);
  for (int i = 0; i < n; ++i) {
    SahTri& t = tri[i];
    for (int k = 0; k < 3; ++k) { t.lo[k] = INFINITY; t.hi[k] = -INFINITY; }
    for (int v = 0; v < 3; ++v)
      for (int k = 0; k < 3; ++k) {
        const float x = V[3 * (int64_t)T[3 * (int64_t)i + v] + k];
        t.lo[k] = fminf(t.lo[k], x);
        t.hi[k] = fmaxf(t.hi[k], x);
      }
    for (int k = 0; k < 3; ++k) t.c[k] = 0.5f * (t.lo[k] + t.hi[k]);
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  child.assign(n - 1, make_int2(0, 0));
  par_int.assign(n - 1, -1);
  par_leaf.assign(n, -1);
  struct Job { int b, e, node; };
  std::vector<Job> stack;
  stack.push_back({0, n, 0});
  int next = 1;
  while (!stack.empty()) {
    const Job j = stack.back();
    stack.pop_back();
    const int cnt = j.e - j.b;
    float cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = j.b; i < j.e; ++i)
      for (int k = 0; k < 3; ++k) {
        cmin[k] = fminf(cmin[k], tri[idx[i]].c[k]);
        cmax[k] = fmaxf(cmax[k], tri[idx[i]].c[k]);
      }
    int ax = 0;
    for (int k = 1; k < 3; ++k)
      if (cmax[k] - cmin[k] > cmax[ax] - cmin[ax]) ax = k;
    const float ext = cmax[ax] - cmin[ax];
    int mid = j.b + cnt / 2;
    if (ext > 0.f) {
      Box3 bb[kBins];
      int bc[kBins] = {0};
      const float sc = kBins / ext;
      auto bin_of = [&](int t) { return std::min(kBins - 1, std::max(0, (int)((tri[t].c[ax] - cmin[ax]) * sc))); };
      for (int i = j.b; i < j.e; ++i) {
        const int b = bin_of(idx[i]);
        bb[b].grow(tri[idx[i]].lo, tri[idx[i]].hi);
        ++bc[b];
      }
      float right_area[kBins];
      int right_cnt[kBins];
      Box3 acc;
      int ac = 0;
      for (int b = kBins - 1; b > 0; --b) {
        acc.grow(bb[b].lo, bb[b].hi);
        ac += bc[b];
        right_area[b] = acc.area();
        right_cnt[b] = ac;
      }
      Box3 la;
      int lc = 0, best = -1;
      float best_cost = INFINITY;
      for (int b = 0; b < kBins - 1; ++b) {  // split between bins b and b + 1
        la.grow(bb[b].lo, bb[b].hi);
        lc += bc[b];
        if (lc == 0 || right_cnt[b + 1] == 0) continue;
        const float cost = la.area() * lc + right_area[b + 1] * right_cnt[b + 1];
        if (cost < best_cost) { best_cost = cost; best = b; }
      }
      if (best >= 0) {
        int* m = std::partition(idx.data() + j.b, idx.data() + j.e, [&](int t) { return bin_of(t) <= best; });
        mid = (int)(m - idx.data());
      }
    }
    if (mid <= j.b || mid >= j.e) {  // degenerate split: median by centroid
      mid = j.b + cnt / 2;
      std::nth_element(idx.data() + j.b, idx.data() + mid, idx.data() + j.e,
                       [&](int a, int b) { return tri[a].c[ax] < tri[b].c[ax]; });
    }
    int2 ch;
    // push the right child first so that the left one is numbered (and laid out) next
    if (j.e - mid == 1) {
      ch.y = ~mid;
      par_leaf[mid] = j.node;
    } else {
      ch.y = -1;  // filled below
    }
    if (mid - j.b == 1) {
      ch.x = ~j.b;
      par_leaf[j.b] = j.node;
    } else {
      ch.x = next++;
      par_int[ch.x] = j.node;
    }
    if (j.e - mid > 1) {
      ch.y = next++;
      par_int[ch.y] = j.node;
      stack.push_back({mid, j.e, ch.y});
    }
    if (mid - j.b > 1) stack.push_back({j.b, mid, ch.x});
    child[j.node] = ch;
  }
  keys.resize(n);
  for (int i = 0; i < n; ++i) keys[i] = (unsigned long long)(unsigned)idx[i];
}
}  // namespace

cudaError_t build_bvh(const float* V, const int32_t* T, const float* hV, const int32_t* hT, int sah,
                      const float* mu, const uint8_t* fl, int32_t n,
                      float4** tri32, float** triv, int32_t** tri_prim, float** tri_mu,
                      uint8_t** tri_flags, double4_32a** tri_plane, float** tri_inv_n, BvhNode** nodes, int32_t* root,
                      cudaStream_t st) {
  int n_pow2 = 1;
  while (n_pow2 < n) n_pow2 <<= 1;
  int n_int = n > 1 ? n - 1 : 1;
  CK(cudaMalloc(tri32, sizeof(float4) * 3 * n));
  CK(cudaMalloc(triv, sizeof(float) * 9 * n));
  CK(cudaMalloc(tri_prim, sizeof(int32_t) * n));
  CK(cudaMalloc(tri_mu, sizeof(float) * n));
  CK(cudaMalloc(tri_flags, n));
  CK(cudaMalloc(tri_plane, (sizeof(double4_32a) + 2 * sizeof(float4)) * n));  // FP64 planes, then FP32 pairs
  CK(cudaMalloc(tri_inv_n, sizeof(float) * n));
  CK(cudaMalloc(nodes, sizeof(BvhNode) * n_int));
  float* bb;
  unsigned long long* keys;
  int2* child;
  int *par_int, *par_leaf, *flags;
  float4 *lbl, *lbh, *ibl, *ibh;
  CK(cudaMalloc(&bb, 6 * sizeof(float)));
  CK(cudaMalloc(&keys, sizeof(unsigned long long) * n_pow2));
  CK(cudaMalloc(&child, sizeof(int2) * n_int));
  CK(cudaMalloc(&par_int, sizeof(int) * n_int));
  CK(cudaMalloc(&par_leaf, sizeof(int) * n));
  CK(cudaMalloc(&flags, sizeof(int) * n_int));
  CK(cudaMalloc(&lbl, sizeof(float4) * n));
  CK(cudaMalloc(&lbh, sizeof(float4) * n));
  CK(cudaMalloc(&ibl, sizeof(float4) * n_int));
  CK(cudaMalloc(&ibh, sizeof(float4) * n_int));
  float init[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  CK(cudaMemcpyAsync(bb, init, sizeof(init), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(flags, 0, sizeof(int) * n_int, st));
  CK(cudaMemsetAsync(par_leaf, 0xff, sizeof(int) * n, st));
  const int B = 256;
  std::vector<unsigned long long> h_keys;
  std::vector<int2> h_child;
  std::vector<int> h_par_int, h_par_leaf;
  if (sah && n > 1) {
    // hierarchy and leaf order from the host SAH build
    sah_build(hV, hT, n, h_keys, h_child, h_par_int, h_par_leaf);
    CK(cudaMemcpyAsync(keys, h_keys.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(child, h_child.data(), sizeof(int2) * (n - 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(par_int, h_par_int.data(), sizeof(int) * (n - 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(par_leaf, h_par_leaf.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  } else {
    // Morton order (30-bit keys, bitonic sort) and the Karras hierarchy on the device
    k_bounds<<<(int)ceil_div(n, B) < 1024 ? (int)ceil_div(n, B) : 1024, B, 0, st>>>(V, T, n, bb);
    k_morton<<<(int)ceil_div(n_pow2, B), B, 0, st>>>(V, T, n, n_pow2, bb, keys);
    for (int k = 2; k <= n_pow2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1)
        k_bitonic<<<(int)ceil_div(n_pow2, B), B, 0, st>>>(keys, n_pow2, k, j);
  }
  k_leaves<<<(int)ceil_div(n, B), B, 0, st>>>(V, T, mu, fl, keys, n, lbl, lbh, *tri32, *triv, *tri_prim,
                                               *tri_mu, *tri_flags, *tri_plane, *tri_inv_n);
  if (n > 1) {
    if (!(sah && n > 1)) k_hierarchy<<<(int)ceil_div(n - 1, B), B, 0, st>>>(keys, n, child, par_int, par_leaf);
    k_refit<<<(int)ceil_div(n, B), B, 0, st>>>(n, child, par_int, par_leaf, lbl, lbh, ibl, ibh, flags);
  } else {
    k_single<<<1, 1, 0, st>>>(child);
  }
  k_pack<<<(int)ceil_div(n_int, B), B, 0, st>>>(n_int, child, lbl, lbh, ibl, ibh, *nodes);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  *root = 0;
  cudaFree(bb);
  cudaFree(keys);
  cudaFree(child);
  cudaFree(par_int);
  cudaFree(par_leaf);
  cudaFree(flags);
  cudaFree(lbl);
  cudaFree(lbh);
  cudaFree(ibl);
  cudaFree(ibh);
  return cudaSuccess;
}

}  // namespace sonar
