// Element-echo synthesis on the 5th-generation tensor cores.
//
// With element phasors separable, exp(j k_a u.p_m) = ey[mx] ez[my], the echoes of a
// tile of T consecutive range samples are one complex contraction over the hits k:
//   S[n][my nx + mx] = sum_k (g_k(n) ey_k[mx]) ez_k[my],  g_k(n) = c_k R(t_n - tau_k),
// i.e. D[(n, mx)][(my, re/im)] = A[(n, mx)][(k, re/im)] . B[(k, re/im)][(my, re/im)]
// with T nx = 128 rows (the MMA M), 2 ny columns (N) and two K columns per hit; B is
// the real 4-form of ez (row (my, 0) = (Re ez, -Im ez), row (my, 1) = (Im ez, Re ez)).
//
// Persistent CTAs take equal contiguous ranges of the delay-sorted hits and walk them
// in K-blocks of up to 32 hits whose taps fall inside at most TMAX tiles. Sixteen
// generator warps stage each K-block (taps from the pulse table, phasors by sincospi),
// write the B operand and one A operand per touched tile straight into shared memory
// in the UMMA 128-byte-swizzle K-major layout (BF16; FP32 form also the residual lo
// parts), one thread issues tcgen05.mma into a ring of TMEM accumulators (one per
// tile), and four epilogue warps add a tile's accumulator into S (FP32, vector
// atomics) once the walk has passed it. The FP32 form runs three BF16 passes per
// operand pair (hi*hi, hi*lo, lo*hi).
#include <limits.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace sonar {
namespace {
using namespace tc;

constexpr int KH = 32;           // hits per K-block: K = 64 BF16 columns (re, im)
constexpr int NA = 3;            // A operand ring slots (hi + lo)
constexpr int NB = 2;            // B operand ring slots (hi + lo)
constexpr int RING = 8;          // TMEM accumulator slots of 64 columns
constexpr int TMAX = 5;          // tiles one K-block may touch
constexpr int kGenWarps = 16;
constexpr int kEpiWarp0 = 1;     // warps 1..4: epilogue, warp 0: MMA, warps 5..20: generators
constexpr int kGenWarp0 = 5;
constexpr int kThreadsTC = 32 * (kGenWarp0 + kGenWarps);
constexpr int kGenThreads = 32 * kGenWarps;
constexpr int A_BYTES = 128 * 128;  // 128 rows x 64 BF16
constexpr int B_BYTES = 64 * 128;   // up to 64 rows x 64 BF16
constexpr int kMaxAx = 64;

template <int WT>
struct Stage {
  HitRec rec[KH];
  int n[KH];
  float2 g[WT][KH];        // tap-major: staging writes and operand reads are conflict-free
  float2 ey[KH][kMaxAx];   // element-major per hit: a warp reads 32 consecutive elements
  float2 ez[KH][kMaxAx];
};

template <int WT>
constexpr size_t tc_smem_bytes() {
  return 1024 + (size_t)NA * 2 * A_BYTES + (size_t)NB * 2 * B_BYTES + 2 * sizeof(Stage<WT>) + 64 * 8 + 64;
}

struct KBlk {
  int cnt, t_first, t_last;
};

// First-tap rows of the 32 sorted hits from h (lane i holds hit h + i; INT_MAX past the
// end). Loaded one K-block ahead so the latency overlaps the current K-block's work.
__device__ __forceinline__ int load_window(const int32_t* ng, int64_t h, int64_t h_end, int lane) {
  const int64_t idx = h + lane;
  return idx < h_end ? __ldg(&ng[idx]) : INT_MAX;
}

// K-block starting at the window's first hit: as many hits (<= 32) as keep every tap
// inside TMAX tiles of T rows. Warp-cooperative (all 32 lanes), identical in every role.
__device__ __forceinline__ KBlk kblock_from(int v, int T, int W) {
  const int g0 = __shfl_sync(0xffffffffu, v, 0);
  KBlk k;
  k.t_first = g0 / T;
  const int limit = T * (k.t_first + TMAX) - W;
  const unsigned ok = __ballot_sync(0xffffffffu, v <= limit);
  k.cnt = __popc(ok);
  if (k.cnt < 1) k.cnt = 1;  // cannot happen for W <= T (TMAX - 1) + 1
  const int g_last = __shfl_sync(0xffffffffu, v, k.cnt - 1);
  k.t_last = (g_last + W - 1) / T;
  return k;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_lo(float a, float b, uint32_t hi) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&hi);
  float2 f = __bfloat1622float2(h);
  return pack_bf16(a - f.x, b - f.y);
}
__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void red_add2(float* dst, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(dst), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void gen_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kGenThreads) : "memory"); }

#define TMEM_LD_16(taddr, r)                                                                                  \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), \
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),         \
                 "=r"(r[15])                                                                                   \
               : "r"(taddr))

// Bounded wait that gives up for good once any role of the CTA has timed out.
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
  if (*abort_flag) return false;
  if (mbar_wait(bar, parity, err)) return true;
  *abort_flag = 1;
  return false;
}

template <int WT>
__global__ void __launch_bounds__(kThreadsTC, 1) k_synth_tc(SynthArgs a, uint32_t idesc) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;                              // NA x (hi, lo)
  uint8_t* sB = sA + NA * 2 * A_BYTES;             // NB x (hi, lo)
  Stage<WT>* st = reinterpret_cast<Stage<WT>*>(sB + NB * 2 * B_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(st + 2);
  uint64_t* a_full = bars;
  uint64_t* a_empty = bars + NA;
  uint64_t* b_full = bars + 2 * NA;
  uint64_t* b_empty = bars + 2 * NA + NB;
  uint64_t* tdone = bars + 2 * NA + 2 * NB;
  uint64_t* tfree = tdone + RING;
  uint64_t* done = tfree + RING;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = a.nx, ny = a.ny, M = nx * ny;
  const int T = 128 / nx;
  const int W = a.taps;
  const int n_brows = 2 * ny;
  const int64_t H = *a.n_valid;
  const int64_t h0 = H * blockIdx.x / gridDim.x, h1 = H * (blockIdx.x + 1) / gridDim.x;
  const bool fp32_form = a.n_pass == 3;

  __shared__ float2 s_rtab[kRTabS + 5];
  for (int i = threadIdx.x; i < kRTabS + 5; i += blockDim.x) s_rtab[i] = a.rtab_s[i];
  if (threadIdx.x == 0) {
    for (int i = 0; i < NA; ++i) { mbar_init(smem_u32(&a_full[i]), kGenWarps); mbar_init(smem_u32(&a_empty[i]), 1); }
    for (int i = 0; i < NB; ++i) { mbar_init(smem_u32(&b_full[i]), kGenWarps); mbar_init(smem_u32(&b_empty[i]), 1); }
    for (int i = 0; i < RING; ++i) { mbar_init(smem_u32(&tdone[i]), 1); mbar_init(smem_u32(&tfree[i]), 4); }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(RING * 64) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------- MMA issuer
    int uses[RING];
    for (int i = 0; i < RING; ++i) uses[i] = 0;
    int live_lo = INT_MAX, live_hi = -1, j = 0, a_idx = 0;
    int win = load_window(a.sorted_n, h0, h1, lane);
    for (int64_t h = h0; h < h1;) {
      const KBlk kb = kblock_from(win, T, W);
      const int64_t hn = h + kb.cnt;
      win = load_window(a.sorted_n, hn, h1, lane);
      if (lane == 0) {
        // tiles the walk has passed: their accumulators are final once these MMAs land
        for (int u = live_lo; u <= live_hi && u < kb.t_first; ++u) tc_commit(smem_u32(&tdone[u % RING]));
        const int bslot = j % NB;
        const bool b_ok = wait_or_abort(smem_u32(&b_full[bslot]), (j / NB) & 1, abort_flag, a.err);
        for (int t = kb.t_first; t <= kb.t_last; ++t) {
          const int slot = t % RING;
          const bool fresh = t > live_hi;
          bool ok = b_ok;
          if (fresh) {
            const int use = uses[slot]++;
            if (use > 0) ok = ok && wait_or_abort(smem_u32(&tfree[slot]), (use - 1) & 1, abort_flag, a.err);
          }
          const int aslot = a_idx % NA;
          ok = ok && wait_or_abort(smem_u32(&a_full[aslot]), (a_idx / NA) & 1, abort_flag, a.err);
          if (ok) {
            tc_fence_after();
            const uint32_t d = tmem_base + (uint32_t)(slot * 64);
            const uint32_t ah = smem_u32(sA + aslot * 2 * A_BYTES), al = ah + A_BYTES;
            const uint32_t bh = smem_u32(sB + bslot * 2 * B_BYTES), bl = bh + B_BYTES;
            for (int pass = 0; pass < a.n_pass; ++pass) {
              const uint32_t aa = pass == 2 ? al : ah, bb = pass == 1 ? bl : bh;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                tc_mma(d, sw128_desc(aa + kk * 32), sw128_desc(bb + kk * 32), idesc,
                       (fresh && pass == 0 && kk == 0) ? 0u : 1u);
            }
            tc_commit(smem_u32(&a_empty[aslot]));
          }
          ++a_idx;
        }
        if (b_ok) tc_commit(smem_u32(&b_empty[bslot]));
      }
      // live tiles: from this K-block's first tile to the furthest tile touched so far
      live_lo = kb.t_first;
      if (kb.t_last > live_hi) live_hi = kb.t_last;
      ++j;
      h = hn;
      __syncwarp();
    }
    if (lane == 0) {
      for (int u = live_lo; u <= live_hi; ++u) tc_commit(smem_u32(&tdone[u % RING]));
      tc_commit(smem_u32(done));
      mbar_wait(smem_u32(done), 0, a.err);
    }
    __syncwarp();
  } else if (warp < kGenWarp0) {
    // ------------------------------------------------------------- epilogue
    const int q = warp & 3;
    const int L = q * 32 + lane;
    const int nl = L / nx, mx = L - nl * nx;
    int uses[RING], cur[RING];
    for (int i = 0; i < RING; ++i) { uses[i] = 0; cur[i] = 0; }
    int live_lo = INT_MAX, live_hi = -1;
    auto flush = [&](int u) {
      const int slot = u % RING;
      const bool ok = wait_or_abort(smem_u32(&tdone[slot]), cur[slot] & 1, abort_flag, a.err);
      if (ok) {
        tc_fence_after();
        float* dst = reinterpret_cast<float*>(a.S + (int64_t)(u * T + nl) * M + mx);
        for (int c0 = 0; c0 < n_brows; c0 += 16) {
          uint32_t v[16];
          TMEM_LD_16(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(slot * 64 + c0), v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int my = c0 / 2 + i;
            red_add2(dst + 2 * (int64_t)my * nx, __uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tfree[slot]));
    };
    int win = load_window(a.sorted_n, h0, h1, lane);
    for (int64_t h = h0; h < h1;) {
      const KBlk kb = kblock_from(win, T, W);
      const int64_t hn = h + kb.cnt;
      win = load_window(a.sorted_n, hn, h1, lane);
      for (int u = live_lo; u <= live_hi && u < kb.t_first; ++u) flush(u);
      for (int t = (live_hi + 1 > kb.t_first ? live_hi + 1 : kb.t_first); t <= kb.t_last; ++t) cur[t % RING] = uses[t % RING]++;
      live_lo = kb.t_first;
      if (kb.t_last > live_hi) live_hi = kb.t_last;
      h = hn;
    }
    for (int u = live_lo; u <= live_hi; ++u) flush(u);
  } else {
    // ------------------------------------------------------------- operand generators
    const int gt = threadIdx.x - kGenWarp0 * 32;
    const int lnx = 31 - __clz(nx);  // nx is a power of two
    int j = 0, a_idx = 0;
    // hit records are fetched one K-block ahead: 32 records from the K-block's first hit
    // (one coalesced 16-byte load per thread; records past the K-block are ignored)
    auto fetch_recs = [&](int64_t hs) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      const int64_t k = hs + (gt >> 1);
      if (gt < 2 * KH && k < h1) v = __ldg(reinterpret_cast<const uint4*>(a.hits_sorted + k) + (gt & 1));
      return v;
    };
    int win = load_window(a.sorted_n, h0, h1, lane);
    uint4 recv = fetch_recs(h0);
    for (int64_t h = h0; h < h1;) {
      const KBlk kb = kblock_from(win, T, W);
      const int64_t hn = h + kb.cnt;
      win = load_window(a.sorted_n, hn, h1, lane);
      Stage<WT>& S = st[j & 1];
      if (gt < 2 * KH) reinterpret_cast<uint4*>(&S.rec[gt >> 1])[gt & 1] = recv;
      recv = fetch_recs(hn);
      gen_bar();
      // taps c_k R((u0 + i) dt) from the pulse table; padding hits contribute zero
      for (int item = gt; item < KH * WT; item += kGenThreads) {
        const int k = item & (KH - 1), q = item >> 5;
        const bool valid = k < kb.cnt;
        const HitRec& hr = S.rec[k];
        float2 g = make_float2(0.f, 0.f);
        if (valid && q < W) {
          // 4-point Lagrange interpolation in the shared-memory table (error ~4e-8)
          const float x = (hr.u0 + (float)q) * a.rtab_s_scale + (float)(kRTabS / 2 + 2);
          if (x >= 1.0f && x < (float)(kRTabS + 3)) {
            const int i = (int)x;
            const float f = x - (float)i;
            const float wm = -f * (f - 1.f) * (f - 2.f) * (1.f / 6.f);
            const float w0 = (f + 1.f) * (f - 1.f) * (f - 2.f) * 0.5f;
            const float w1 = -(f + 1.f) * f * (f - 2.f) * 0.5f;
            const float w2 = (f + 1.f) * f * (f - 1.f) * (1.f / 6.f);
            const float2 r0 = s_rtab[i - 1], r1 = s_rtab[i], r2 = s_rtab[i + 1], r3 = s_rtab[i + 2];
            const float rr = wm * r0.x + w0 * r1.x + w1 * r2.x + w2 * r3.x;
            const float ri = wm * r0.y + w0 * r1.y + w1 * r2.y + w2 * r3.y;
            g = make_float2(hr.cr * rr - hr.ci * ri, hr.cr * ri + hr.ci * rr);
          }
        }
        S.g[q][k] = g;
        if (q == 0) S.n[k] = valid ? hr.nglob : INT_MIN / 2;
      }
      // separable element phasors ey[mx] = exp(j 2 pi (d/lambda) (mx - (nx-1)/2) u_y), ez likewise
      for (int item = gt; item < KH * nx; item += kGenThreads) {
        const int mx = item & (nx - 1), k = item >> lnx;
        float2 e = make_float2(0.f, 0.f);
        if (k < kb.cnt) {
          float s, c;
          sincospif(2.0f * a.pitch_over_lambda * ((float)mx - 0.5f * (float)(nx - 1)) * S.rec[k].uy, &s, &c);
          e = make_float2(c, s);
        }
        S.ey[k][mx] = e;
      }
      for (int item = gt; item < KH * ny; item += kGenThreads) {
        const int k = item / ny, my = item - k * ny;
        float2 e = make_float2(0.f, 0.f);
        if (k < kb.cnt) {
          float s, c;
          sincospif(2.0f * a.pitch_over_lambda * ((float)my - 0.5f * (float)(ny - 1)) * S.rec[k].uz, &s, &c);
          e = make_float2(c, s);
        }
        S.ez[k][my] = e;
      }
      gen_bar();
      // B operand: rows (my, re/im), K = (hit, re/im); a warp covers 32 rows of one chunk
      const int bslot = j % NB;
      wait_or_abort(smem_u32(&b_empty[bslot]), ((j / NB) & 1) ^ 1, abort_flag, a.err);
      {
        const uint32_t bh = smem_u32(sB + bslot * 2 * B_BYTES), bl = bh + B_BYTES;
        for (int idx = gt; idx < n_brows * 8; idx += kGenThreads) {
          const int c = idx / n_brows, row = idx - c * n_brows;
          const int my = row >> 1, r = row & 1;
          uint32_t hv[4], lv[4];
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const float2 e = S.ez[4 * c + kk][my];
            const float x = r == 0 ? e.x : e.y, y = r == 0 ? -e.y : e.x;
            hv[kk] = pack_bf16(x, y);
            lv[kk] = pack_lo(x, y, hv[kk]);
          }
          const uint32_t off = (uint32_t)(row * 128 + ((c ^ (row & 7)) << 4));
          sts128(bh + off, hv[0], hv[1], hv[2], hv[3]);
          if (fp32_form) sts128(bl + off, lv[0], lv[1], lv[2], lv[3]);
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&b_full[bslot]));
      // A operand per touched tile: rows (n, mx), K = (hit, re/im); a warp covers 32
      // consecutive rows of one 16-byte chunk (conflict-free under the 128-byte swizzle)
      for (int t = kb.t_first; t <= kb.t_last; ++t) {
        const int aslot = a_idx % NA;
        wait_or_abort(smem_u32(&a_empty[aslot]), ((a_idx / NA) & 1) ^ 1, abort_flag, a.err);
        const uint32_t ah = smem_u32(sA + aslot * 2 * A_BYTES), al = ah + A_BYTES;
        for (int idx = gt; idx < 128 * 8; idx += kGenThreads) {
          const int c = idx >> 7, row = idx & 127;
          const int nl = row >> lnx, mx = row & (nx - 1);
          const int trow = t * T + nl;
          uint32_t hv[4], lv[4];
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const int k = 4 * c + kk;
            const int tap = trow - S.n[k];
            float x = 0.f, y = 0.f;
            if (tap >= 0 && tap < WT) {
              const float2 g = S.g[tap][k], e = S.ey[k][mx];
              x = g.x * e.x - g.y * e.y;
              y = g.x * e.y + g.y * e.x;
            }
            hv[kk] = pack_bf16(x, y);
            lv[kk] = pack_lo(x, y, hv[kk]);
          }
          const uint32_t off = (uint32_t)(row * 128 + ((c ^ (row & 7)) << 4));
          sts128(ah + off, hv[0], hv[1], hv[2], hv[3]);
          if (fp32_form) sts128(al + off, lv[0], lv[1], lv[2], lv[3]);
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&a_full[aslot]));
        ++a_idx;
      }
      ++j;
      h = hn;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(RING * 64) : "memory");
  }
}

}  // namespace

bool synth_tc_supported(int nx, int ny, int taps) {
  const bool pow2 = nx >= 4 && nx <= 64 && (nx & (nx - 1)) == 0;
  return pow2 && ny % 8 == 0 && ny >= 8 && ny <= 32 && taps <= 16 && taps <= (128 / nx) * (TMAX - 1) + 1;
}

cudaError_t prepare_synth_tc() {
  cudaError_t e = cudaFuncSetAttribute(k_synth_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes<8>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_synth_tc<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes<12>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_synth_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes<16>());
}

cudaError_t launch_synth_tc(const SynthArgs& a, int sm_count, cudaStream_t st) {
  const uint32_t idesc = make_idesc(1, 128, 2 * a.ny);
  if (a.taps <= 8) k_synth_tc<8><<<sm_count, kThreadsTC, tc_smem_bytes<8>(), st>>>(a, idesc);
  else if (a.taps <= 12) k_synth_tc<12><<<sm_count, kThreadsTC, tc_smem_bytes<12>(), st>>>(a, idesc);
  else k_synth_tc<16><<<sm_count, kThreadsTC, tc_smem_bytes<16>(), st>>>(a, idesc);
  return cudaGetLastError();
}

}  // namespace sonar
