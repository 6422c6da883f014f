// Learned echo surrogate: a per-beam 1-D convolutional network (Sec. II.B proposes learned
// scattering functions in place of costly echo physics) that maps a cheap geometric
// rendering of each beam to the coherent envelope the plain method forms.
//
// Network: six convolutions along range, kernel 9, zero padding at the beam's ends,
// channels 4 -> 64 -> 64 -> 64 -> 64 -> 64 -> 1, ReLU after the first five. Weights are
// BF16 (rounded from FP32 master copies), accumulation FP32, activations and
// back-propagated gradients stored as BF16 between layers, biases FP32.
//
// Activation buffers hold one beam per rb = n_range + 16 rows of 64 BF16 channels (128
// bytes per row): 8 zero rows, the n_range bins, 8 zero rows. The zero rows are the
// convolution's padding and are never written.
//
// Kernels:
//  - k_sur_input: layer 0 from the rendering. The input is sparse (two hits per beam,
//    each splatted onto two bins), so each position sums the few taps that touch it.
//  - k_conv<MODE>: a hidden 64 -> 64 layer as an implicit GEMM on tcgen05. M = 128
//    positions, N = 64 output channels, K = 9 taps x 64 input channels. The 136 input
//    rows a tile needs are staged once by TMA (128-byte swizzle); tap k reads them
//    through a matrix descriptor that starts k rows later (36 MMAs of K = 16 per tile).
//    The weights of all taps stay in shared memory. MODE 0 is the forward layer (bias,
//    ReLU); MODE 1 the backward-data pass (the transposed, tap-reversed weights, and the
//    previous layer's ReLU mask).
//  - k_dw: a hidden layer's weight gradient dW_k[o][c] = sum_p dz[p][o] x[p + k - 4][c]
//    on tcgen05. M = 128 = (tap parity, output channel): tensor memory holds the dz
//    window as the A operand, rows 64..127 shifted one position, so one MMA makes two
//    taps; B is the staged input tile read K-rows-shifted per tap pair (MN-major). Five
//    tap pairs accumulate in five TMEM accumulators over the CTA's whole range of
//    positions, then add into the gradient.
//  - k_sur_head / k_sur_head_bwd: the 64 -> 1 output layer (warp-shuffle reductions),
//    the loss gradient, and its backward pass.
//  - k_sur_l1_dw: layer 0's gradient from the sparse input.
//  - k_sur_pack: Adam (Kingma & Ba 2015) and the BF16 weight copies.
//  - k_cmp_*: the metrics that compare a surrogate volume with the plain method's.
#include <limits.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace sonar {
namespace {
using namespace tc;

constexpr int C = kSurC;
constexpr int KT = kSurK;
constexpr int HALO = kSurHalo;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
  if (*abort_flag) return false;
  if (mbar_wait(bar, parity, err)) return true;
  *abort_flag = 1;
  return false;
}

// K-major 128-byte-swizzle descriptor of an operand whose first row is `row` rows past a
// 1024-byte-aligned stage (rows of 128 bytes, 8-row swizzle atoms 1024 bytes apart). The
// start address alone carries the shift: the tensor cores take each row's swizzle phase
// from its shared-memory address bits, so the matrix base-offset field stays zero
// (measured: a base offset equal to the start row's phase in the atom scrambles the
// operand; zero matches the FP64 reference to rounding).
__device__ __forceinline__ uint64_t shifted_desc(uint32_t stage, int row, uint32_t extra_bytes) {
  return sw128_desc(stage + (uint32_t)row * 128u + extra_bytes);
}
// The same for an MN-major operand (128-byte rows along MN, K down the rows): 8-row K
// groups 1024 bytes apart; the MN-group stride is unused for N = 64.
__device__ __forceinline__ uint64_t shifted_desc_mn(uint32_t stage, int row) {
  const uint32_t addr = stage + (uint32_t)row * 128u;
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(1024 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t base, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols) : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ----------------------------------------------------------------- parameters
__global__ void k_sur_pack(SurNet n, int update, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= kSurParams) return;
  float th = n.theta[i];
  if (update) {
    const float g = n.grad[i];
    const float m = b1 * n.m[i] + (1.f - b1) * g;
    const float v = b2 * n.v[i] + (1.f - b2) * g * g;
    n.m[i] = m;
    n.v[i] = v;
    th -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    n.theta[i] = th;
  }
  int l = 0;
  int64_t off = 0;
  for (; l < 5; ++l) {
    const int64_t next = off + (int64_t)sur_cout(l) * sur_cin(l) * KT + sur_cout(l);
    if (i < next) break;
    off = next;
  }
  const int64_t r = i - off;
  if (r >= (int64_t)sur_cout(l) * sur_cin(l) * KT) return;  // a bias: read from theta
  const int k = (int)(r % KT), ci = (int)((r / KT) % sur_cin(l)), co = (int)(r / (KT * sur_cin(l)));
  const __nv_bfloat16 h = __float2bfloat16_rn(th);
  if (l == 0) {
    n.w_in[r] = __bfloat162float(h);
  } else if (l == 5) {
    n.w_out[ci * KT + k] = __bfloat162float(h);
  } else {
    const int L = l - 1;
    n.wf[((int64_t)(L * KT + k) * C + co) * C + ci] = h;
    n.wb[((int64_t)(L * KT + (KT - 1 - k)) * C + ci) * C + co] = h;
  }
}

// ----------------------------------------------------------------- layer 0
// One thread per (selected beam, bin, group of 8 channels): a warp writes four whole
// 128-byte rows per store. A hit at one-way length L sits at bin coordinate
// x = (L - r_min) / dr - 1/2 and splats 1 - f, f onto bins floor(x), floor(x) + 1.
// Channels: 0 first-hit splat, 1 second-hit splat, 2 incidence cosine, 3 reflectivity
// (both hits, as their splats' amplitudes). Most bins see no splat within the kernel's
// reach and get the bias alone.
__global__ void __launch_bounds__(256) k_sur_input(const float* feat, const int32_t* beams, int64_t i0, int64_t n_feat,
                                                   int nr, double r_min, double inv_dr, const float* w_in,
                                                   const float* b_in, __nv_bfloat16* act, int rb, int* err) {
  // grid: x over (bin, channel group) of one beam, y over beams
  // the beam's splat positions, in FP64 once per block (FP64 work per thread is slow
  // on this part): first bin and fraction of each hit, n0 = INT_MIN for no hit
  __shared__ int s_n0[2];
  __shared__ float s_fr[2];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = t & 7;  // channels 8 g .. 8 g + 7
  const int p = t >> 3;
  const int64_t i = i0 + blockIdx.y;
  const int64_t beam = beams ? (int64_t)beams[i] : i;
  const bool valid = beam >= 0 && beam < n_feat;
  const float4* f4 = reinterpret_cast<const float4*>(feat + (valid ? beam : 0) * 8);
  if (threadIdx.x < 2) {
    const float L = __ldg(&f4[threadIdx.x]).x;
    int n0 = INT_MIN;
    float fr = 0.f;
    if (valid && L > 0.f) {
      const double x = ((double)L - r_min) * inv_dr - 0.5;
      const double fl = floor(x);
      n0 = (int)fl;
      fr = (float)(x - fl);
    }
    s_n0[threadIdx.x] = n0;
    s_fr[threadIdx.x] = fr;
  }
  __syncthreads();
  float z[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) z[c] = __ldg(&b_in[8 * g + c]);
  if (!valid) {
    if (g == 0 && p == 0) atomicOr(err, kErrIndex);
  } else {
    for (int h = 0; h < 2; ++h) {
      const int n0 = s_n0[h];
      if (n0 == INT_MIN) continue;
      if (n0 + 1 < p - KT / 2 || n0 > p + KT / 2) continue;  // no splat reaches this bin
      const float4 f = __ldg(&f4[h]);
      const float fr = s_fr[h];
      for (int e = 0; e < 2; ++e) {
        const int q = n0 + e;
        const int k = q - p + KT / 2;
        if (q < 0 || q >= nr || k < 0 || k >= KT) continue;
        const float w = e ? fr : 1.f - fr;
        const float v2 = f.y * w, v3 = f.z * w;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float* wc = w_in + (8 * g + c) * 4 * KT + k;
          z[c] += __ldg(wc + h * KT) * w + __ldg(wc + 2 * KT) * v2 + __ldg(wc + 3 * KT) * v3;
        }
      }
    }
  }
  uint4* dst = reinterpret_cast<uint4*>(act + ((int64_t)i * rb + HALO + p) * C) + g;
  *dst = make_uint4(pack_bf16(fmaxf(z[0], 0.f), fmaxf(z[1], 0.f)), pack_bf16(fmaxf(z[2], 0.f), fmaxf(z[3], 0.f)),
                    pack_bf16(fmaxf(z[4], 0.f), fmaxf(z[5], 0.f)), pack_bf16(fmaxf(z[6], 0.f), fmaxf(z[7], 0.f)));
}

// ----------------------------------------------------------------- hidden layers (tcgen05)
constexpr int kConvThreads = 192;   // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr int kConvStages = 4;
constexpr int kConvRing = 4;        // TMEM accumulators of 64 columns
constexpr int kStageRows = 128 + KT - 1;
constexpr int kStageBytes = 18432;  // 136 rows x 128 bytes, rounded up to 1 KB
constexpr int kWBytes = KT * C * 128;
constexpr size_t kConvSmem = 1024 + kWBytes + (size_t)kConvStages * kStageBytes + 256;
static_assert(kStageRows * 128 <= kStageBytes, "stage holds a tile and its halo");

template <int MODE>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv(const __grid_constant__ SurConvArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sW = smem;
  uint8_t* sA = smem + kWBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sA + kConvStages * kStageBytes);
  uint64_t* empty = full + kConvStages;
  uint64_t* acc_full = empty + kConvStages;
  uint64_t* acc_empty = acc_full + kConvRing;
  uint64_t* wfull = acc_empty + kConvRing;
  uint64_t* done = wfull + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kConvStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int r = 0; r < kConvRing; ++r) {
      mbar_init(smem_u32(&acc_full[r]), 1);
      mbar_init(smem_u32(&acc_empty[r]), 4);
    }
    mbar_init(smem_u32(wfull), 1);
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, kConvRing * 64);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int64_t t_first = blockIdx.x, t_step = gridDim.x;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- TMA producer
      mbar_expect_tx(smem_u32(wfull), kWBytes);
      for (int k = 0; k < KT; ++k) tma_load_2d(smem_u32(sW + k * C * 128), &a.map_w, 0, k * C, smem_u32(wfull));
      int it = 0;
      for (int64_t t = t_first; t < a.n_tiles; t += t_step, ++it) {
        const int s = it % kConvStages;
        if (it >= kConvStages &&
            !wait_or_abort(smem_u32(&empty[s]), ((it / kConvStages) & 1) ^ 1, abort_flag, a.err))
          break;
        const int64_t beam = t / a.tiles_per_beam;
        const int p0 = (int)(t % a.tiles_per_beam) * 128;
        mbar_expect_tx(smem_u32(&full[s]), kStageRows * 128);
        tma_load_2d(smem_u32(sA + s * kStageBytes), &a.map_x, 0, (int)(beam * a.rb + HALO + p0 - KT / 2),
                    smem_u32(&full[s]));
      }
      // every copy this thread issued has landed before the CTA may exit
      for (int s = 0; s < kConvStages && s < it; ++s) {
        const int last = s + ((it - 1 - s) / kConvStages) * kConvStages;
        mbar_wait(smem_u32(&full[s]), (last / kConvStages) & 1, a.err);
      }
      mbar_wait(smem_u32(wfull), 0, a.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------------------------------------------------- MMA issuer
      const uint32_t idesc = make_idesc(1, 128, 64);
      bool ok = wait_or_abort(smem_u32(wfull), 0, abort_flag, a.err);
      int it = 0;
      const uint32_t wbase = smem_u32(sW);
      for (int64_t t = t_first; ok && t < a.n_tiles; t += t_step, ++it) {
        const int s = it % kConvStages, r = it % kConvRing;
        if (!wait_or_abort(smem_u32(&full[s]), (it / kConvStages) & 1, abort_flag, a.err)) break;
        if (it >= kConvRing && !wait_or_abort(smem_u32(&acc_empty[r]), ((it / kConvRing) & 1) ^ 1, abort_flag, a.err))
          break;
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(r * 64);
        const uint32_t abase = smem_u32(sA + s * kStageBytes);
#pragma unroll 1
        for (int k = 0; k < KT; ++k) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            tc_mma(d, shifted_desc(abase, k, kk * 32), sw128_desc(wbase + k * C * 128 + kk * 32), idesc,
                   (k | kk) ? 1u : 0u);
        }
        tc_commit(smem_u32(&empty[s]));
        tc_commit(smem_u32(&acc_full[r]));
      }
      tc_commit(smem_u32(done));
      mbar_wait(smem_u32(done), 0, a.err);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lane quarter of this warp
    int it = 0;
    for (int64_t t = t_first; t < a.n_tiles; t += t_step, ++it) {
      const int r = it % kConvRing;
      if (!wait_or_abort(smem_u32(&acc_full[r]), (it / kConvRing) & 1, abort_flag, a.err)) break;
      tc_fence_after();
      uint32_t v0[32], v1[32];
      const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(r * 64);
      TMEM_LD_32(ta, v0);
      TMEM_LD_32(ta + 32, v1);
      tmem_ld_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acc_empty[r]));
      const int64_t beam = t / a.tiles_per_beam;
      const int p = (int)(t % a.tiles_per_beam) * 128 + q * 32 + lane;
      const int64_t row = beam * a.rb + HALO + p;
      uint4* dst = reinterpret_cast<uint4*>(a.out + row * C);
      float f[C];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        f[c] = __uint_as_float(v0[c]);
        f[32 + c] = __uint_as_float(v1[c]);
      }
      if (MODE == 0) {
#pragma unroll
        for (int c = 0; c < C; ++c) f[c] = fmaxf(f[c] + __ldg(&a.bias[c]), 0.f);
      } else {
        const uint4* mk = reinterpret_cast<const uint4*>(a.mask + row * C);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint4 m = __ldg(&mk[j]);
          const uint32_t mw[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (!(bf_lo(mw[e]) > 0.f)) f[8 * j + 2 * e] = 0.f;
            if (!(bf_hi(mw[e]) > 0.f)) f[8 * j + 2 * e + 1] = 0.f;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j)
        dst[j] = make_uint4(pack_bf16(f[8 * j], f[8 * j + 1]), pack_bf16(f[8 * j + 2], f[8 * j + 3]),
                            pack_bf16(f[8 * j + 4], f[8 * j + 5]), pack_bf16(f[8 * j + 6], f[8 * j + 7]));
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_free(tmem_base, kConvRing * 64);
}

// ----------------------------------------------------------------- hidden-layer weight gradient
constexpr int kDwThreads = 192;        // warp 0 TMA, warp 1 MMA, warps 2..5 dz window + epilogue
constexpr int kDwStages = 4;
constexpr int kDwRows = 80;            // staged rows per K-block: positions q0 - 8 .. q0 + 71
constexpr int kDwTile = kDwRows * 128; // 10240 bytes, a multiple of 1 KB
constexpr int kDwPairs = 5;            // tap pairs (0,1) .. (8, -)
constexpr int kDwAcol = kDwPairs * 64; // TMEM columns of the five accumulators; A windows follow
constexpr size_t kDwSmem = 1024 + (size_t)kDwStages * 2 * kDwTile + 256;

__global__ void __launch_bounds__(kDwThreads, 1) k_dw(const __grid_constant__ SurDwArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sX = smem;                          // [stage] input rows
  uint8_t* sZ = smem + kDwStages * kDwTile;    // [stage] dz rows
  uint64_t* full = reinterpret_cast<uint64_t*>(sZ + kDwStages * kDwTile);
  uint64_t* empty = full + kDwStages;
  uint64_t* a_full = empty + kDwStages;
  uint64_t* a_empty = a_full + 2;
  uint64_t* done = a_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kDwStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1 + 4);  // the MMA's commit and the four window warps
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&a_full[i]), 4);
      mbar_init(smem_u32(&a_empty[i]), 1);
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int64_t kb0 = a.n_kb * blockIdx.x / gridDim.x, kb1 = a.n_kb * (blockIdx.x + 1) / gridDim.x;
  const int nkb = (int)(kb1 - kb0);

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (; it < nkb; ++it) {
        const int s = it % kDwStages;
        if (it >= kDwStages && !wait_or_abort(smem_u32(&empty[s]), ((it / kDwStages) & 1) ^ 1, abort_flag, a.err))
          break;
        const int64_t kb = kb0 + it;
        const int64_t beam = kb / a.kb_per_beam;
        const int q0 = (int)(kb % a.kb_per_beam) * 64;
        const int row = (int)(beam * a.rb + HALO + q0 - 8);
        mbar_expect_tx(smem_u32(&full[s]), 2 * kDwTile);
        tma_load_2d(smem_u32(sX + s * kDwTile), &a.map_x, 0, row, smem_u32(&full[s]));
        tma_load_2d(smem_u32(sZ + s * kDwTile), &a.map_dz, 0, row, smem_u32(&full[s]));
      }
      // every copy this thread issued has landed before the CTA may exit
      for (int s = 0; s < kDwStages && s < it; ++s) {
        const int last = s + ((it - 1 - s) / kDwStages) * kDwStages;
        mbar_wait(smem_u32(&full[s]), (last / kDwStages) & 1, a.err);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc(1, 128, 64) | (1u << 16);  // B MN-major
      for (int it = 0; it < nkb; ++it) {
        const int s = it % kDwStages, slot = it & 1;
        if (!wait_or_abort(smem_u32(&full[s]), (it / kDwStages) & 1, abort_flag, a.err)) break;
        if (!wait_or_abort(smem_u32(&a_full[slot]), (it >> 1) & 1, abort_flag, a.err)) break;
        tc_fence_after();
        const uint32_t xb = smem_u32(sX + s * kDwTile);
        const uint32_t at = tmem_base + (uint32_t)(kDwAcol + slot * 32);
#pragma unroll 1
        for (int j = 0; j < kDwPairs; ++j) {
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            // B[c][kappa] = x[q0 + 16 ks + kappa + 2 j - 4][c]: stage row 4 + 2 j + 16 ks
            const int row = 4 + 2 * j + 16 * ks;
            tc_mma_tmem_a(tmem_base + (uint32_t)(j * 64), at + (uint32_t)(ks * 8), shifted_desc_mn(xb, row),
                          idesc, (it == 0 && ks == 0) ? 0u : 1u);
          }
        }
        tc_commit(smem_u32(&empty[s]));
        tc_commit(smem_u32(&a_empty[slot]));
      }
      tc_commit(smem_u32(done));
    }
  } else {
    // ------------------------------------------- dz windows into TMEM, then the epilogue
    const int q = warp & 3;
    const int m = q * 32 + lane;     // TMEM lane: (tap parity t, output channel o)
    const int t = m >> 6, o = m & 63;
    float db = 0.f;
    for (int it = 0; it < nkb; ++it) {
      const int s = it % kDwStages, slot = it & 1;
      if (!wait_or_abort(smem_u32(&full[s]), (it / kDwStages) & 1, abort_flag, a.err)) break;
      if (it >= 2 && !wait_or_abort(smem_u32(&a_empty[slot]), ((it >> 1) & 1) ^ 1, abort_flag, a.err)) break;
      tc_fence_after();
      const int64_t kb = kb0 + it;
      const int q0 = (int)(kb % a.kb_per_beam) * 64;
      const uint8_t* z = sZ + s * kDwTile;
      // column c holds positions kappa = 2c, 2c + 1 of dz[q0 + kappa - t]: stage row 8 + kappa - t
      uint32_t cols[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        float v[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int kap = 2 * c + e, row = 8 + kap - t, p = q0 + kap - t;
          const uint16_t raw = *reinterpret_cast<const uint16_t*>(z + row * 128 + ((((o >> 3) ^ (row & 7))) << 4) +
                                                                  (o & 7) * 2);
          v[e] = (p >= 0 && p < a.nr) ? __uint_as_float((uint32_t)raw << 16) : 0.f;
        }
        if (t == 0) db += v[0] + v[1];
        cols[c] = pack_bf16(v[0], v[1]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[s]));  // this warp is done with the dz rows
      const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(kDwAcol + slot * 32);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const uint32_t w8[8] = {cols[8 * g], cols[8 * g + 1], cols[8 * g + 2], cols[8 * g + 3],
                                cols[8 * g + 4], cols[8 * g + 5], cols[8 * g + 6], cols[8 * g + 7]};
        tmem_st8(ta + (uint32_t)(8 * g), w8);
      }
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&a_full[slot]));
    }
    if (t == 0) atomicAdd(&a.grad_b[o], db);
    const bool ok = !*abort_flag && mbar_wait(smem_u32(done), 0, a.err);
    if (ok && nkb > 0) {
      tc_fence_after();
#pragma unroll
      for (int j = 0; j < kDwPairs; ++j) {
        const int k = 2 * j + t;
        uint32_t v0[32], v1[32];
        const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(j * 64);
        TMEM_LD_32(ta, v0);
        TMEM_LD_32(ta + 32, v1);
        tmem_ld_wait();
        if (k < KT) {
          float* gw = a.grad_w + (int64_t)o * C * KT + k;
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            atomicAdd(gw + c * KT, __uint_as_float(v0[c]));
            atomicAdd(gw + (32 + c) * KT, __uint_as_float(v1[c]));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    // the MMA's last commit has arrived before the accumulators are released
    if (lane == 0) mbar_wait(smem_u32(done), 0, a.err);
    __syncwarp();
    tmem_free(tmem_base, 512);
  }
}

// ----------------------------------------------------------------- output layer
// One warp per 64 consecutive bins of a beam; lane l holds input channels 2l, 2l + 1.
// Every lane accumulates its channels' share of all 64 outputs from the 72 rows they
// read (so that many loads are in flight), then a halving shuffle reduction leaves the
// outputs of bins p0 + l and p0 + 32 + l in lane l.
constexpr int kHeadBins = 64;
__global__ void __launch_bounds__(256) k_sur_head(const __nv_bfloat16* act5, const float* w_out, const float* b_out,
                                                  int64_t n_sel, int nr, int rb, const float* target,
                                                  const int32_t* beams, int64_t n_feat, float inv_scale, float g_scale,
                                                  float* g, double* loss, float* env_out, float e_scale, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int wpb = nr / kHeadBins;
  const int64_t i = wg / wpb;
  if (i >= n_sel) return;
  const int p0 = (int)(wg % wpb) * kHeadBins;
  float wa[KT], wb[KT];
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    wa[k] = __ldg(&w_out[(2 * lane) * KT + k]);
    wb[k] = __ldg(&w_out[(2 * lane + 1) * KT + k]);
  }
  const uint32_t* base = reinterpret_cast<const uint32_t*>(act5 + ((int64_t)i * rb + HALO + p0 - KT / 2) * C);
  float acc[kHeadBins];
#pragma unroll
  for (int j = 0; j < kHeadBins; ++j) acc[j] = 0.f;
#pragma unroll
  for (int r = 0; r < kHeadBins + KT - 1; ++r) {
    const uint32_t u = __ldg(&base[r * (C / 2) + lane]);
    const float x0 = bf_lo(u), x1 = bf_hi(u);
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const int j = r - k;  // row p0 - 4 + r feeds bin p0 + j through tap k
      if (j >= 0 && j < kHeadBins) acc[j] = fmaf(wa[k], x0, fmaf(wb[k], x1, acc[j]));
    }
  }
  // bins j and j + 32 reduce side by side: after the five halving steps lane l holds the
  // sums of bins l (acc[0]) and 32 + l (acc[32])
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
      for (int j = 0; j < s; ++j) {
        float* a = acc + 32 * half;
        const float send = up ? a[j] : a[j + s];
        const float keep = up ? a[j + s] : a[j];
        a[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
      }
    }
  }
  const float b5 = __ldg(b_out);
  float sq = 0.f;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const float yhat = acc[32 * half] + b5;
    const int p = p0 + 32 * half + lane;
    const int64_t idx = i * nr + p;
    if (target) {
      const int64_t beam = beams ? (int64_t)beams[i] : i;
      float d = 0.f;
      if (beam < 0 || beam >= n_feat) {
        if (lane == 0) atomicOr(err, kErrIndex);
      } else {
        d = yhat - __ldg(&target[beam * nr + p]) * inv_scale;
      }
      g[idx] = g_scale * d;
      sq += d * d;
    }
    if (env_out) env_out[idx] = e_scale * yhat;
  }
  if (target) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) atomicAdd(loss, (double)sq);
  }
}

// Backward of the output layer over 256 bins of a beam: dz5[p][c] = [a5[p][c] > 0]
// sum_k W5[c][k] g[p - k + 4] (one thread per bin), and the partial sums of
// dW5[c][k] = sum_p a5[p][c] g[p - k + 4] and db5 = sum_p g[p] (one thread per entry).
__global__ void __launch_bounds__(256) k_sur_head_bwd(const __nv_bfloat16* act5, const float* g, const float* w_out,
                                                      int nr, int rb, __nv_bfloat16* dz5, float* grad_w5,
                                                      float* grad_b5) {
  __shared__ float sg[256 + KT - 1];
  __shared__ __align__(16) uint32_t sa[256 * C / 2];
  __shared__ float sw[C * KT];
  __shared__ float red[8];
  const int chunks = nr / 256;
  const int64_t i = blockIdx.x / chunks;
  const int p0 = (int)(blockIdx.x % chunks) * 256;
  const int t = threadIdx.x;
  for (int j = t; j < 256 + KT - 1; j += 256) {
    const int p = p0 - KT / 2 + j;
    sg[j] = (p >= 0 && p < nr) ? g[i * nr + p] : 0.f;
  }
  const uint4* src = reinterpret_cast<const uint4*>(act5 + ((int64_t)i * rb + HALO + p0) * C);
  uint4* sa4 = reinterpret_cast<uint4*>(sa);
  for (int j = t; j < 256 * C / 8; j += 256) sa4[j] = __ldg(&src[j]);
  for (int j = t; j < C * KT; j += 256) sw[j] = w_out[j];
  __syncthreads();
  {
    const int p = p0 + t;
    uint32_t out[C / 2];
#pragma unroll
    for (int c2 = 0; c2 < C / 2; ++c2) {
      const uint32_t u = sa[t * (C / 2) + c2];
      float d[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = 2 * c2 + e;
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < KT; ++k) s = fmaf(sw[c * KT + k], sg[t - k + 2 * (KT / 2)], s);
        d[e] = ((e ? bf_hi(u) : bf_lo(u)) > 0.f) ? s : 0.f;
      }
      out[c2] = pack_bf16(d[0], d[1]);
    }
    uint4* dst = reinterpret_cast<uint4*>(dz5 + ((int64_t)i * rb + HALO + p) * C);
#pragma unroll
    for (int j = 0; j < 8; ++j) dst[j] = make_uint4(out[4 * j], out[4 * j + 1], out[4 * j + 2], out[4 * j + 3]);
  }
  for (int e = t; e < C * KT; e += 256) {
    const int c = e / KT, k = e % KT;
    float s = 0.f;
    for (int u = 0; u < 256; ++u) {
      const uint32_t w = sa[u * (C / 2) + (c >> 1)];
      s = fmaf((c & 1) ? bf_hi(w) : bf_lo(w), sg[u - k + 2 * (KT / 2)], s);
    }
    atomicAdd(&grad_w5[e], s);
  }
  float gs = sg[t + KT / 2];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gs += __shfl_xor_sync(0xffffffffu, gs, o);
  if ((t & 31) == 0) red[t >> 5] = gs;
  __syncthreads();
  if (t == 0) {
    float s = 0.f;
    for (int w = 0; w < 8; ++w) s += red[w];
    atomicAdd(grad_b5, s);
  }
}

// Layer-0 gradients, one block of 64 threads (output channels) per selected beam:
// dW0[o][c][k] = sum over the beam's splat bins q of x0[q][c] dz1[q - k + 4][o], and
// db0[o] = sum_p dz1[p][o].
__global__ void __launch_bounds__(64) k_sur_l1_dw(const float* feat, const int32_t* beams, int64_t n_feat, int nr,
                                                  double r_min, double inv_dr, const __nv_bfloat16* dz1, int rb,
                                                  float* grad_w0, float* grad_b0) {
  const int64_t i = blockIdx.x;
  const int o = threadIdx.x;
  const int64_t beam = beams ? (int64_t)beams[i] : i;
  const __nv_bfloat16* col = dz1 + (int64_t)i * rb * C + o;
  float db = 0.f;
  for (int p = 0; p < nr; ++p) db += __bfloat162float(col[(int64_t)(HALO + p) * C]);
  atomicAdd(&grad_b0[o], db);
  if (beam < 0 || beam >= n_feat) return;  // flagged by the forward kernels
  float acc[4][KT];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int k = 0; k < KT; ++k) acc[c][k] = 0.f;
  const float4* f4 = reinterpret_cast<const float4*>(feat + beam * 8);
  for (int h = 0; h < 2; ++h) {
    const float4 f = f4[h];
    if (!(f.x > 0.f)) continue;
    const double x = ((double)f.x - r_min) * inv_dr - 0.5;
    const double fl = floor(x);
    const int n0 = (int)fl;
    const float fr = (float)(x - fl);
    for (int e = 0; e < 2; ++e) {
      const int q = n0 + e;
      if (q < 0 || q >= nr) continue;
      const float w = e ? fr : 1.f - fr;
#pragma unroll
      for (int k = 0; k < KT; ++k) {
        const float d = __bfloat162float(col[(int64_t)(HALO + q - k + KT / 2) * C]);  // halo rows are zero
        acc[h][k] += w * d;
        acc[2][k] += f.y * w * d;
        acc[3][k] += f.z * w * d;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int k = 0; k < KT; ++k)
      if (acc[c][k] != 0.f) atomicAdd(&grad_w0[(o * 4 + c) * KT + k], acc[c][k]);
}

// ----------------------------------------------------------------- geometric envelope
// The rendering turned into an envelope without the network, one thread per (beam, bin):
// E[n] = TVG(r_n) sum_h a_h |R(t_n - 2 L_h / c)|, a_h = Gamma_h^2 sqrt(mu_h kappa_h
// dOmega_b) / L_h exp(-2 alpha L_h), dOmega_b the beam cell's solid angle; R from the
// pulse-autocorrelation table (entry i at u = -T + 2 T i / n_tab), interpolated linearly.
__global__ void __launch_bounds__(256) k_sur_geometric(const float* feat, int64_t n_beams, int nba, int nbe,
                                                       double hfov, double vfov, int nr, double r_min, double dr,
                                                       double two_inv_c, double alpha, double T, double tab_scale,
                                                       const float2* rtab, int n_tab, float* env) {
  // one thread per (beam, bin); FP64 only for the delay difference (multiplies and adds:
  // the reciprocals two_inv_c = 2 / c_ref and tab_scale = n_tab / (2 T) come from the host)
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= n_beams * nr) return;
  const int64_t b = gid / nr;
  const int n = (int)(gid % nr);
  const int j = (int)((b % ((int64_t)nba * nbe)) / nba);
  const float del = (float)(vfov / nbe), el_lo = (float)(-vfov / 2) + j * del;
  const float domega = (float)(hfov / nba) * (sinf(el_lo + del) - sinf(el_lo));
  const double r = r_min + (n + 0.5) * dr;
  const double t = r * two_inv_c;
  const float4* f4 = reinterpret_cast<const float4*>(feat + b * 8);
  float e = 0.f;
  for (int h = 0; h < 2; ++h) {
    const float4 f = f4[h];
    if (!(f.x > 0.f)) continue;
    const double u = t - (double)f.x * two_inv_c;
    if (!(fabs(u) < T)) continue;
    const double x = (u + T) * tab_scale;
    int i = (int)floor(x);
    if (i >= n_tab) i = n_tab - 1;
    const float w = (float)(x - i);
    const float2 a = __ldg(&rtab[i]), c = __ldg(&rtab[i + 1]);
    const float re = a.x + w * (c.x - a.x), im = a.y + w * (c.y - a.y);
    const float amp = f.w * f.w * sqrtf(f.z * f.y * domega) / f.x * expf(-2.f * (float)alpha * f.x);
    e += amp * sqrtf(re * re + im * im);
  }
  env[gid] = e * (float)r * expf(2.f * (float)alpha * (float)r);
}

// ----------------------------------------------------------------- comparison metrics
// Pass 1, one warp per (ping, beam): squared error and reference energy (totals[0..1]),
// the peak bin of each volume at or beyond n_blank (first index on ties), the beam's
// reference maximum and the ping's.
__global__ void __launch_bounds__(256) k_cmp_pass1(const float* env, const float* ref, int64_t n_beams, int nb, int nr,
                                                   int n_blank, unsigned* ping_max, int32_t* beam_pk, float* beam_max,
                                                   double* totals) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_beams) return;
  const float* e = env + w * nr;
  const float* r = ref + w * nr;
  double se = 0.0, sr = 0.0;
  unsigned long long ke = 0, kr = 0;
  float mr = 0.f;
  for (int n = lane; n < nr; n += 32) {
    const float a = e[n], b = r[n];
    se += (double)(a - b) * (a - b);
    sr += (double)b * b;
    if (n >= n_blank) {
      // (value bits, bin complement): the largest key is the largest value, then the lowest bin
      const unsigned long long ka = ((unsigned long long)__float_as_uint(fmaxf(a, 0.f)) << 32) | (0xFFFFFFFFu - n);
      const unsigned long long kb = ((unsigned long long)__float_as_uint(fmaxf(b, 0.f)) << 32) | (0xFFFFFFFFu - n);
      ke = ka > ke ? ka : ke;
      kr = kb > kr ? kb : kr;
      mr = fmaxf(mr, b);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    se += __shfl_xor_sync(0xffffffffu, se, o);
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    const unsigned long long xe = __shfl_xor_sync(0xffffffffu, ke, o), xr = __shfl_xor_sync(0xffffffffu, kr, o);
    ke = xe > ke ? xe : ke;
    kr = xr > kr ? xr : kr;
    mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
  }
  if (lane == 0) {
    atomicAdd(&totals[0], se);
    atomicAdd(&totals[1], sr);
    beam_pk[2 * w] = (int32_t)(0xFFFFFFFFu - (uint32_t)(ke & 0xFFFFFFFFu));
    beam_pk[2 * w + 1] = (int32_t)(0xFFFFFFFFu - (uint32_t)(kr & 0xFFFFFFFFu));
    beam_max[w] = mr;
    atomicMax(&ping_max[w / nb], __float_as_uint(mr));
  }
}

// Pass 2: beams whose reference peak reaches rel of the ping maximum (lit beams) add
// |peak bin - reference peak bin| (totals[2] sum, [3] count, [4] within 1 bin, [5] within
// 4 bins); cells whose reference reaches rel of the ping maximum add the intensity
// moments of both volumes ([6] count, [7] sum I, [8] sum I^2, [9] sum I_ref,
// [10] sum I_ref^2).
__global__ void __launch_bounds__(256) k_cmp_pass2(const float* env, const float* ref, int64_t n_beams, int nb, int nr,
                                                   float rel, const unsigned* ping_max, const int32_t* beam_pk,
                                                   const float* beam_max, double* totals) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_beams) return;
  const float thr = rel * __uint_as_float(ping_max[w / nb]);
  const float* e = env + w * nr;
  const float* r = ref + w * nr;
  double n = 0, s1 = 0, s2 = 0, r1 = 0, r2 = 0;
  for (int k = lane; k < nr; k += 32) {
    const float b = r[k];
    if (b >= thr && b > 0.f) {
      const double ia = (double)e[k] * e[k], ib = (double)b * b;
      n += 1;
      s1 += ia;
      s2 += ia * ia;
      r1 += ib;
      r2 += ib * ib;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(0xffffffffu, n, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    r1 += __shfl_xor_sync(0xffffffffu, r1, o);
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  }
  if (lane == 0) {
    if (beam_max[w] >= thr && beam_max[w] > 0.f) {
      const int d = abs(beam_pk[2 * w] - beam_pk[2 * w + 1]);
      atomicAdd(&totals[2], (double)d);
      atomicAdd(&totals[3], 1.0);
      if (d <= 1) atomicAdd(&totals[4], 1.0);
      if (d <= 4) atomicAdd(&totals[5], 1.0);
    }
    if (n > 0) {
      atomicAdd(&totals[6], n);
      atomicAdd(&totals[7], s1);
      atomicAdd(&totals[8], s2);
      atomicAdd(&totals[9], r1);
      atomicAdd(&totals[10], r2);
    }
  }
}

}  // namespace

cudaError_t sur_pack(const SurNet& n, int update, float lr, float b1, float b2, float eps, float bc1, float bc2,
                     cudaStream_t st) {
  k_sur_pack<<<(unsigned)ceil_div(kSurParams, 256), 256, 0, st>>>(n, update, lr, b1, b2, eps, bc1, bc2);
  return cudaGetLastError();
}

cudaError_t sur_input(const float* feat, const int32_t* beams, int64_t n_sel, int64_t n_feat, int nr, double r_min,
                      double inv_dr, const SurNet& n, __nv_bfloat16* act1, int rb, int* err, cudaStream_t st) {
  // nr is a multiple of 256: whole blocks per beam; beams in launches of at most 65535
  for (int64_t i0 = 0; i0 < n_sel; i0 += 65535) {
    const unsigned ny = (unsigned)(n_sel - i0 < 65535 ? n_sel - i0 : 65535);
    k_sur_input<<<dim3((unsigned)(nr * 8 / 256), ny), 256, 0, st>>>(feat, beams, i0, n_feat, nr, r_min, inv_dr, n.w_in,
                                                                     n.theta + sur_boff(0), act1, rb, err);
  }
  return cudaGetLastError();
}

cudaError_t sur_conv_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_conv<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConvSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConvSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwSmem);
  return e;
}

cudaError_t sur_conv(const SurConvArgs& a, bool backward, int sm_count, cudaStream_t st) {
  if (a.n_tiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)(a.n_tiles < sm_count ? a.n_tiles : sm_count);
  if (backward) k_conv<1><<<grid, kConvThreads, kConvSmem, st>>>(a);
  else k_conv<0><<<grid, kConvThreads, kConvSmem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t sur_head(const __nv_bfloat16* act5, const SurNet& n, int64_t n_sel, int nr, int rb, const float* target,
                     const int32_t* beams, int64_t n_feat, float inv_scale, float g_scale, float* g, double* loss,
                     float* env_out, float e_scale, int* err, cudaStream_t st) {
  const int64_t warps = n_sel * (nr / kHeadBins);
  if (warps == 0) return cudaSuccess;
  k_sur_head<<<(unsigned)ceil_div(warps * 32, 256), 256, 0, st>>>(act5, n.w_out, n.theta + sur_boff(5), n_sel, nr, rb,
                                                                   target, beams, n_feat, inv_scale, g_scale, g, loss,
                                                                   env_out, e_scale, err);
  return cudaGetLastError();
}

cudaError_t sur_head_bwd(const __nv_bfloat16* act5, const float* g, const SurNet& n, int64_t n_sel, int nr, int rb,
                         __nv_bfloat16* dz5, cudaStream_t st) {
  const int64_t blocks = n_sel * (nr / 256);
  if (blocks == 0) return cudaSuccess;
  k_sur_head_bwd<<<(unsigned)blocks, 256, 0, st>>>(act5, g, n.w_out, nr, rb, dz5, n.grad + sur_woff(5),
                                                   n.grad + sur_boff(5));
  return cudaGetLastError();
}

cudaError_t sur_dw(const SurDwArgs& a, int sm_count, cudaStream_t st) {
  if (a.n_kb == 0) return cudaSuccess;
  const unsigned grid = (unsigned)(a.n_kb < sm_count ? a.n_kb : sm_count);
  k_dw<<<grid, kDwThreads, kDwSmem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t sur_l1_dw(const float* feat, const int32_t* beams, int64_t n_sel, int64_t n_feat, int nr, double r_min,
                      double inv_dr, const __nv_bfloat16* dz1, int rb, const SurNet& n, cudaStream_t st) {
  if (n_sel == 0) return cudaSuccess;
  k_sur_l1_dw<<<(unsigned)n_sel, 64, 0, st>>>(feat, beams, n_feat, nr, r_min, inv_dr, dz1, rb, n.grad + sur_woff(0),
                                               n.grad + sur_boff(0));
  return cudaGetLastError();
}

cudaError_t sur_geometric(const float* feat, int64_t n_beams, int nba, int nbe, double hfov, double vfov, int nr,
                          double r_min, double dr, double c_ref, double alpha, double T, const float2* rtab, int n_tab,
                          float* env, cudaStream_t st) {
  const int64_t total = n_beams * nr;
  if (total == 0) return cudaSuccess;
  k_sur_geometric<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(feat, n_beams, nba, nbe, hfov, vfov, nr, r_min, dr,
                                                                   2.0 / c_ref, alpha, T, n_tab / (2.0 * T), rtab, n_tab,
                                                                   env);
  return cudaGetLastError();
}

cudaError_t sur_compare(const float* env, const float* ref, int P, int nb, int nr, int n_blank, float rel_thr,
                        unsigned* ping_max, int32_t* beam_pk, float* beam_max, double* totals, cudaStream_t st) {
  const int64_t beams = (int64_t)P * nb;
  const unsigned grid = (unsigned)ceil_div(beams * 32, 256);
  k_cmp_pass1<<<grid, 256, 0, st>>>(env, ref, beams, nb, nr, n_blank, ping_max, beam_pk, beam_max, totals);
  k_cmp_pass2<<<grid, 256, 0, st>>>(env, ref, beams, nb, nr, rel_thr, ping_max, beam_pk, beam_max, totals);
  return cudaGetLastError();
}

}  // namespace sonar
