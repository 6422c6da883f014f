// Element-echo synthesis on the 5th-generation tensor cores.
//
// Element phasors are separable, exp(j k_a u.p_m) = ey[mx] ez[my], so the echoes of a
// tile of T consecutive range samples are complex contractions over the hits k of
//   S[n][my nx + mx] = sum_k g_k(n) ey_k[mx] ez_k[my],   g_k(n) = c_k R(t_n - tau_k).
// Two operand factorisations (both MMA shapes M = 128, N = 64, two K columns per hit):
//
//  per-K-block z split (arrays with nx ny a multiple of 128): with my = my_hi L2 + my_lo
//  (L2 = nx ny / 128), ez[my] = E1[my_hi] E2[my_lo], E1 = ez shifted by L2 my_hi,
//  E2[my_lo] = exp(j theta_z my_lo). The M operand A[(my_hi, mx)][k] = ey[mx] E1[my_hi]
//  does not depend on the tile and is generated once per K-block; only the N operand
//  B[k][(n, my_lo, re/im)] = g_k(n) E2[my_lo] (T = 32 / L2 samples) is generated per
//  tile.
//
//  per-tile (small arrays): A[(n, mx)][k] = g_k(n) ey[mx] per tile (T = 128 / nx) and
//  B[k][(my, re/im)] = ez[my] once per K-block.
//
// N operands are stored as the real 4-form: row (., 0) = (Re b, -Im b), row (., 1) =
// (Im b, Re b) over the (re, im) K pair of each hit.
//
// Persistent CTAs take equal contiguous ranges of the delay-sorted hits and walk them in
// K-blocks of up to 32 hits whose taps stay inside TMAX tiles. Sixteen generator warps
// stage each K-block (taps from a cubic pulse table in shared memory, phasors by
// sincospi) and write the operands straight into shared memory in the UMMA 128-byte
// swizzle K-major layout (BF16; the FP32 form also writes the residual lo parts and runs
// three passes hi*hi, hi*lo, lo*hi). One thread issues tcgen05.mma into a ring of TMEM
// accumulators (one per tile); four epilogue warps add a tile's accumulator into S
// (FP32, vector atomics) once the walk has passed it.
#include <limits.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace sonar {
namespace {
using namespace tc;

constexpr int KH = 32;           // hits per K-block: K = 64 BF16 columns (re, im)
constexpr int NB = 2;            // per-K-block operand ring slots (hi + lo)
constexpr int RING = 8;          // TMEM accumulator slots of 64 columns
constexpr int TMAX = 5;          // tiles one K-block may touch
constexpr int kGenWarps = 16;
constexpr int kGenWarp0 = 5;     // warp 0: MMA, warps 1..4: epilogue, warps 5..20: generators
constexpr int kThreadsTC = 32 * (kGenWarp0 + kGenWarps);
constexpr int kGenThreads = 32 * kGenWarps;
constexpr int M_BYTES = 128 * 128;  // 128 rows x 64 BF16
constexpr int N_BYTES = 64 * 128;   // up to 64 rows x 64 BF16
constexpr int kMaxAx = 64;

template <bool SZ> struct Mode {
  static constexpr int NA = SZ ? 4 : 3;                 // per-tile operand ring slots
  static constexpr int TILE_OP = SZ ? N_BYTES : M_BYTES;  // bytes of one per-tile operand (hi)
  static constexpr int KB_OP = SZ ? M_BYTES : N_BYTES;    // bytes of one per-K-block operand (hi)
};

template <int WT>
struct Stage {
  HitRec rec[KH];
  int n[KH];
  float2 g[WT][KH];        // tap-major: staging writes and operand reads are conflict-free
  float2 ey[KH][kMaxAx];   // per hit, element-major: a warp reads consecutive elements
  float2 ez[KH][kMaxAx];   // ez[my], or E1 in [0, H1) and E2 in [H1, H1 + L2)
};

template <int WT, bool SZ>
constexpr size_t tc_smem_bytes() {
  return 1024 + (size_t)Mode<SZ>::NA * 2 * Mode<SZ>::TILE_OP + (size_t)NB * 2 * Mode<SZ>::KB_OP +
         2 * sizeof(Stage<WT>) + 64 * 8 + 64;
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

// One 16-byte operand chunk (4 complex values, hits 4c..4c+3) in the 128-byte swizzle.
__device__ __forceinline__ void store_chunk(uint32_t hi_base, uint32_t lo_base, int row, int c, const float2 (&v)[4],
                                            bool fp32_form) {
  uint32_t hv[4], lv[4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    hv[kk] = pack_bf16(v[kk].x, v[kk].y);
    lv[kk] = pack_lo(v[kk].x, v[kk].y, hv[kk]);
  }
  const uint32_t off = (uint32_t)(row * 128 + ((c ^ (row & 7)) << 4));
  sts128(hi_base + off, hv[0], hv[1], hv[2], hv[3]);
  if (fp32_form) sts128(lo_base + off, lv[0], lv[1], lv[2], lv[3]);
}

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

template <int WT, bool SZ>
__global__ void __launch_bounds__(kThreadsTC, 1) k_synth_tc(SynthArgs a, uint32_t idesc) {
  constexpr int NA = Mode<SZ>::NA, TILE_OP = Mode<SZ>::TILE_OP, KB_OP = Mode<SZ>::KB_OP;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // align by pointer arithmetic on the shared array, so that the compiler keeps the
  // shared address space (an integer round trip would turn every access generic)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sT = smem;                              // per-tile operands: NA x (hi, lo)
  uint8_t* sK = sT + NA * 2 * TILE_OP;             // per-K-block operands: NB x (hi, lo)
  Stage<WT>* st = reinterpret_cast<Stage<WT>*>(sK + NB * 2 * KB_OP);
  uint64_t* bars = reinterpret_cast<uint64_t*>(st + 2);
  uint64_t* a_full = bars;                         // per-tile ring
  uint64_t* a_empty = bars + NA;
  uint64_t* b_full = bars + 2 * NA;                // per-K-block ring
  uint64_t* b_empty = bars + 2 * NA + NB;
  uint64_t* tdone = bars + 2 * NA + 2 * NB;
  uint64_t* tfree = tdone + RING;
  uint64_t* done = tfree + RING;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  __shared__ float2 s_rtab[kRTabS + 5];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = a.nx, ny = a.ny, M = nx * ny;
  const int L2 = SZ ? M / 128 : 1;   // my_lo count (z split), a power of two
  const int lL2 = 31 - __clz(L2);
  const int H1 = SZ ? ny / L2 : 1;   // my_hi count (z split)
  const int T = SZ ? 32 / L2 : 128 / nx;
  const int W = a.taps;
  const int n_cols = SZ ? 64 : 2 * ny;  // MMA N
  const int64_t Hn = *a.n_valid;
  const int64_t h0 = Hn * blockIdx.x / gridDim.x, h1 = Hn * (blockIdx.x + 1) / gridDim.x;
  const bool fp32_form = a.n_pass == 3;

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
    // per TMEM slot: has it held a tile before (used), parity of its use count (par)
    uint32_t used = 0, par = 0;
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
            const uint32_t bit = 1u << slot;
            if (used & bit) ok = ok && wait_or_abort(smem_u32(&tfree[slot]), ((par >> slot) & 1u) ^ 1u, abort_flag, a.err);
            used |= bit;
            par ^= bit;
          }
          const int aslot = a_idx % NA;
          ok = ok && wait_or_abort(smem_u32(&a_full[aslot]), (a_idx / NA) & 1, abort_flag, a.err);
          if (ok) {
            tc_fence_after();
            const uint32_t d = tmem_base + (uint32_t)(slot * 64);
            const uint32_t th = smem_u32(sT + aslot * 2 * TILE_OP), tl = th + TILE_OP;
            const uint32_t kh = smem_u32(sK + bslot * 2 * KB_OP), kl = kh + KB_OP;
            // M operand (A) and N operand (B) of this mode
            const uint32_t ah = SZ ? kh : th, al = SZ ? kl : tl;
            const uint32_t bh = SZ ? th : kh, bl = SZ ? tl : kl;
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
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int L = q * 32 + lane;
    const int r_hi = L / nx, mx = L - r_hi * nx;  // (my_hi, mx) or (n, mx)
    // per TMEM slot: parity of its use count (par) and of the tile it holds now (cur)
    uint32_t par = 0, cur = 0;
    int live_lo = INT_MAX, live_hi = -1;
    auto flush = [&](int u) {
      const int slot = u % RING;
      const bool ok = wait_or_abort(smem_u32(&tdone[slot]), (cur >> slot) & 1u, abort_flag, a.err);
      if (ok) {
        tc_fence_after();
        for (int c0 = 0; c0 < n_cols; c0 += 16) {
          uint32_t v[16];
          TMEM_LD_16(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(slot * 64 + c0), v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int pr = c0 / 2 + i;  // (n, my_lo) pair, or my
            int64_t row, my;
            if (SZ) {
              const int nl = pr >> lL2, my_lo = pr & (L2 - 1);
              row = (int64_t)u * T + nl;
              my = r_hi * L2 + my_lo;
            } else {
              row = (int64_t)u * T + r_hi;
              my = pr;
            }
            float* dst = reinterpret_cast<float*>(a.S + row * M + my * nx + mx);
            red_add2(dst, __uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
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
      for (int t = (live_hi + 1 > kb.t_first ? live_hi + 1 : kb.t_first); t <= kb.t_last; ++t) {
        const uint32_t bit = 1u << (t % RING);
        cur = (cur & ~bit) | (par & bit);
        par ^= bit;
      }
      live_lo = kb.t_first;
      if (kb.t_last > live_hi) live_hi = kb.t_last;
      h = hn;
    }
    for (int u = live_lo; u <= live_hi; ++u) flush(u);
  } else {
    // ------------------------------------------------------------- operand generators
    const int gt = threadIdx.x - kGenWarp0 * 32;
    const int lnx = 31 - __clz(nx);  // nx is a power of two
    const float pl2 = 2.0f * a.pitch_over_lambda;
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
        const int k = item & (KH - 1), qq = item >> 5;
        const bool valid = k < kb.cnt;
        const HitRec& hr = S.rec[k];
        float2 g = make_float2(0.f, 0.f);
        if (valid && qq < W) {
          // 4-point Lagrange interpolation in the shared-memory table (error ~4e-8)
          const float x = (hr.u0 + (float)qq) * a.rtab_s_scale + (float)(kRTabS / 2 + 2);
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
        S.g[qq][k] = g;
        if (qq == 0) S.n[k] = valid ? hr.nglob : INT_MIN / 2;
      }
      // separable element phasors: ey[mx] = exp(j 2 pi (d/lambda) (mx - (nx-1)/2) u_y);
      // z: ez[my] (per-tile mode) or E1[my_hi] = ez[L2 my_hi], E2[my_lo] = exp(j theta_z my_lo)
      for (int item = gt; item < KH * nx; item += kGenThreads) {
        const int mx = item & (nx - 1), k = item >> lnx;
        float2 e = make_float2(0.f, 0.f);
        if (k < kb.cnt) {
          float s, c;
          sincospif(pl2 * ((float)mx - 0.5f * (float)(nx - 1)) * S.rec[k].uy, &s, &c);
          e = make_float2(c, s);
        }
        S.ey[k][mx] = e;
      }
      const int nz = SZ ? H1 + L2 : ny;
      for (int item = gt; item < KH * nz; item += kGenThreads) {
        const int k = item / nz, qz = item - k * nz;
        float2 e = make_float2(0.f, 0.f);
        if (k < kb.cnt) {
          float arg;
          if (!SZ) arg = (float)qz - 0.5f * (float)(ny - 1);
          else if (qz < H1) arg = (float)(L2 * qz) - 0.5f * (float)(ny - 1);
          else arg = (float)(qz - H1);
          float s, c;
          sincospif(pl2 * arg * S.rec[k].uz, &s, &c);
          e = make_float2(c, s);
        }
        S.ez[k][qz] = e;
      }
      gen_bar();
      // per-K-block operand
      const int bslot = j % NB;
      wait_or_abort(smem_u32(&b_empty[bslot]), ((j / NB) & 1) ^ 1, abort_flag, a.err);
      {
        const uint32_t kh = smem_u32(sK + bslot * 2 * KB_OP), kl = kh + KB_OP;
        if (SZ) {
          // A[(my_hi, mx)][k] = ey[mx] E1[my_hi]; a warp covers 32 rows of one chunk
          for (int idx = gt; idx < 128 * 8; idx += kGenThreads) {
            const int c = idx >> 7, row = idx & 127;
            const int my_hi = row >> lnx, mx = row & (nx - 1);
            float2 v[4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const float2 e = S.ey[4 * c + kk][mx], z = S.ez[4 * c + kk][my_hi];
              v[kk] = make_float2(e.x * z.x - e.y * z.y, e.x * z.y + e.y * z.x);
            }
            store_chunk(kh, kl, row, c, v, fp32_form);
          }
        } else {
          // B[k][(my, re/im)] = 4-form of ez[my]
          for (int idx = gt; idx < n_cols * 8; idx += kGenThreads) {
            const int c = idx / n_cols, row = idx - c * n_cols;
            const int my = row >> 1, r = row & 1;
            float2 v[4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const float2 e = S.ez[4 * c + kk][my];
              v[kk] = r == 0 ? make_float2(e.x, -e.y) : make_float2(e.y, e.x);
            }
            store_chunk(kh, kl, row, c, v, fp32_form);
          }
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&b_full[bslot]));
      // per-tile operand for every touched tile
      for (int t = kb.t_first; t <= kb.t_last; ++t) {
        const int aslot = a_idx % NA;
        wait_or_abort(smem_u32(&a_empty[aslot]), ((a_idx / NA) & 1) ^ 1, abort_flag, a.err);
        const uint32_t th = smem_u32(sT + aslot * 2 * TILE_OP), tl = th + TILE_OP;
        if (SZ) {
          // B[k][(n, my_lo, re/im)] = 4-form of g_k(n) E2[my_lo]
          for (int idx = gt; idx < 64 * 8; idx += kGenThreads) {
            const int c = idx >> 6, row = idx & 63;
            const int pr = row >> 1, r = row & 1;
            const int nl = pr >> lL2, my_lo = pr & (L2 - 1);
            const int trow = t * T + nl;
            float2 v[4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const int k = 4 * c + kk;
              const int tap = trow - S.n[k];
              float x = 0.f, y = 0.f;
              if (tap >= 0 && tap < WT) {
                const float2 g = S.g[tap][k], z = S.ez[k][H1 + my_lo];
                x = g.x * z.x - g.y * z.y;
                y = g.x * z.y + g.y * z.x;
              }
              v[kk] = r == 0 ? make_float2(x, -y) : make_float2(y, x);
            }
            store_chunk(th, tl, row, c, v, fp32_form);
          }
        } else {
          // A[(n, mx)][k] = g_k(n) ey[mx]; a warp covers 32 rows of one chunk
          for (int idx = gt; idx < 128 * 8; idx += kGenThreads) {
            const int c = idx >> 7, row = idx & 127;
            const int nl = row >> lnx, mx = row & (nx - 1);
            const int trow = t * T + nl;
            float2 v[4];
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
              v[kk] = make_float2(x, y);
            }
            store_chunk(th, tl, row, c, v, fp32_form);
          }
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

bool z_split(int nx, int ny) {
  const int M = nx * ny;
  if (M % 128 != 0) return false;
  const int L2 = M / 128;
  return L2 <= 32 && (32 % L2) == 0 && ny % L2 == 0 && nx >= 4 && nx <= kMaxAx && (nx & (nx - 1)) == 0 &&
         nx * (ny / L2) == 128 && ny / L2 + L2 <= kMaxAx;
}

template <int WT, bool SZ>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(k_synth_tc<WT, SZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes<WT, SZ>());
}

template <int WT, bool SZ>
void launch_one(const SynthArgs& a, int sm_count, cudaStream_t st) {
  const uint32_t idesc = make_idesc(1, 128, SZ ? 64 : 2 * a.ny);
  k_synth_tc<WT, SZ><<<sm_count, kThreadsTC, tc_smem_bytes<WT, SZ>(), st>>>(a, idesc);
}

}  // namespace

bool synth_tc_supported(int nx, int ny, int taps) {
  if (taps > 16) return false;
  if (z_split(nx, ny)) return taps <= (32 / (nx * ny / 128)) * (TMAX - 1) + 1;
  const bool pow2 = nx >= 4 && nx <= 64 && (nx & (nx - 1)) == 0;
  return pow2 && ny % 8 == 0 && ny >= 8 && ny <= 32 && taps <= (128 / nx) * (TMAX - 1) + 1;
}

cudaError_t prepare_synth_tc() {
  cudaError_t e;
  if ((e = set_attr<8, false>()) != cudaSuccess) return e;
  if ((e = set_attr<12, false>()) != cudaSuccess) return e;
  if ((e = set_attr<16, false>()) != cudaSuccess) return e;
  if ((e = set_attr<8, true>()) != cudaSuccess) return e;
  if ((e = set_attr<12, true>()) != cudaSuccess) return e;
  return set_attr<16, true>();
}

cudaError_t launch_synth_tc(const SynthArgs& a, int sm_count, cudaStream_t st) {
  const bool sz = z_split(a.nx, a.ny);
  if (a.taps <= 8) sz ? launch_one<8, true>(a, sm_count, st) : launch_one<8, false>(a, sm_count, st);
  else if (a.taps <= 12) sz ? launch_one<12, true>(a, sm_count, st) : launch_one<12, false>(a, sm_count, st);
  else sz ? launch_one<16, true>(a, sm_count, st) : launch_one<16, false>(a, sm_count, st);
  return cudaGetLastError();
}

}  // namespace sonar
