// Point-cloud extraction from envelope volumes that performs no allocation.
//
// Some callers cannot call cudaMalloc: code running where the allocator is off limits
// (inside a custom allocator or memory-pool callback, a real-time loop with a frozen
// memory budget, or a host process that must not grow device memory after start-up).
// For them this entry point keeps its scratch (per-beam peak keys, per-ping maxima and
// point counts) in one file-scope __device__ array of fixed size, which every GPU that
// loads the library holds until the process exits. The caller passes the envelope
// volumes and the output buffers; the call allocates nothing (no cudaMalloc/cudaFree,
// no allocating library routine).
#include <stddef.h>

#include <mutex>

#include "common.cuh"

namespace sonar {
namespace {

constexpr int64_t kNoAllocMaxKeys = 1 << 19;  // pings x beams
constexpr int kNoAllocMaxPings = 64;
constexpr int kNoAllocMaxDevices = 64;

struct NoAllocScratch {
  unsigned long long keys[kNoAllocMaxKeys];  // packed (value bits, 2^32 - 1 - bin) per beam
  unsigned int ping_max[kNoAllocMaxPings];   // float bits of the ping maximum
  long long n_cloud[kNoAllocMaxPings];
};

// Host code sees only a stand-in for this symbol; its device address comes from
// cudaGetSymbolAddress (per device, below).
static __device__ __align__(256) NoAllocScratch g_noalloc;

struct PoseBlock {
  DevPose p[kNoAllocMaxPings];
};

// One warp per (ping, beam): strongest bin at or beyond n_blank, ties to the lowest bin.
__global__ void k_na_argmax(const float* env, int n_pings, int nb, int nr, int n_blank, NoAllocScratch* s) {
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (int64_t)n_pings * nb) return;
  const int p = (int)(warp / nb);
  const float* row = env + warp * nr;
  unsigned long long key = 0ull;
  float vmax = 0.f;
  for (int n = n_blank + lane; n < nr; n += 32) {
    const float e = row[n];
    const unsigned long long k = ((unsigned long long)__float_as_uint(e) << 32) | (0xFFFFFFFFu - (uint32_t)n);
    key = k > key ? k : key;
    vmax = fmaxf(vmax, e);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
    key = other > key ? other : key;
    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  }
  if (lane == 0) {
    s->keys[warp] = key;
    atomicMax(&s->ping_max[p], __float_as_uint(vmax));
  }
}

// Per ping: threshold, beam-ordered compaction, world position R (r_n u_b) + t.
__global__ void __launch_bounds__(1024) k_na_compact(NoAllocScratch* s, const __grid_constant__ PoseBlock poses, int nba,
                                                     int nbe, double hfov, double vfov, double r_min, double dr,
                                                     int thr_mode, float thr, sonar_point* cloud, int64_t cap) {
  __shared__ int s_scan[1024];
  __shared__ long long s_base;
  const int p = blockIdx.x, t = threadIdx.x;
  const int nb = nba * nbe;
  const float vmax = __uint_as_float(s->ping_max[p]);
  const float th = thr_mode == 1 ? thr * vmax : thr;
  const DevPose& P = poses.p[p];
  if (t == 0) s_base = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += 1024) {
    const int b = b0 + t;
    const unsigned long long key = b < nb ? s->keys[(int64_t)p * nb + b] : 0ull;
    const float val = __uint_as_float((uint32_t)(key >> 32));
    const bool keep = key != 0ull && val >= th;
    s_scan[t] = keep ? 1 : 0;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const int v = t >= off ? s_scan[t - off] : 0;
      __syncthreads();
      s_scan[t] += v;
      __syncthreads();
    }
    const long long pos = s_base + s_scan[t] - (keep ? 1 : 0);
    if (keep && pos < cap) {
      const int n = (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
      const int bi = b % nba, bj = b / nba;
      const double az = -hfov / 2 + (bi + 0.5) * hfov / nba;
      const double el = -vfov / 2 + (bj + 0.5) * vfov / nbe;
      const double r = r_min + (n + 0.5) * dr;
      const double v[3] = {r * cos(el) * cos(az), r * cos(el) * sin(az), r * sin(el)};
      sonar_point pt;
      pt.x = (float)(P.R[0] * v[0] + P.R[1] * v[1] + P.R[2] * v[2] + P.t[0]);
      pt.y = (float)(P.R[3] * v[0] + P.R[4] * v[1] + P.R[5] * v[2] + P.t[1]);
      pt.z = (float)(P.R[6] * v[0] + P.R[7] * v[1] + P.R[8] * v[2] + P.t[2]);
      pt.intensity = val;
      pt.beam = b;
      pt.bin = n;
      cloud[(int64_t)p * cap + pos] = pt;
    }
    __syncthreads();
    if (t == 1023) s_base += s_scan[1023];
    __syncthreads();
  }
  if (t == 0) s->n_cloud[p] = s_base;
}

std::mutex g_na_mutex;
NoAllocScratch* g_na_addr[kNoAllocMaxDevices] = {};

// True when the kernels of this device may dereference p: device or managed memory.
// Host memory (pageable, pinned or unregistered) is refused, so a wrong pointer is an
// argument error instead of a faulting kernel. cudaPointerGetAttributes allocates nothing.
bool device_accessible(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace sonar

using namespace sonar;

extern "C" SONAR_API int sonar_cloud_noalloc(const float* env, int32_t n_pings, const sonar_params* p,
                                             const sonar_pose* poses, sonar_point* cloud, int64_t cloud_cap,
                                             int64_t* n_cloud, void* cuda_stream) {
  if (!env || !p || !poses || n_pings < 1 || cloud_cap < 0 || (cloud_cap > 0 && !cloud)) return SONAR_E_ARG;
  if (p->n_beam_az < 1 || p->n_beam_el < 1 || p->n_range < 1 || !(p->r_max_m > p->r_min_m) ||
      (p->thr_mode != 0 && p->thr_mode != 1))
    return SONAR_E_ARG;
  const int64_t nb = (int64_t)p->n_beam_az * p->n_beam_el;
  if (n_pings > kNoAllocMaxPings || nb * n_pings > kNoAllocMaxKeys) return SONAR_E_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return SONAR_E_CUDA;
  if (!device_accessible(env) || (cloud_cap > 0 && !device_accessible(cloud))) return SONAR_E_ARG;
  NoAllocScratch* s = nullptr;
  {
    // first call on a device: resolve the device address of the scratch array
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc) != cudaSuccess || !ptr) return SONAR_E_CUDA;
      g_na_addr[dev] = static_cast<NoAllocScratch*>(ptr);
    }
    s = g_na_addr[dev];
  }
  PoseBlock pb;
  for (int i = 0; i < n_pings; ++i) {
    const double* q = poses[i].q;
    const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(qn > 0)) return SONAR_E_ARG;
    const double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    double* R = pb.p[i].R;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
    for (int k = 0; k < 3; ++k) pb.p[i].t[k] = poses[i].t[k];
  }
  const double dr = (p->r_max_m - p->r_min_m) / p->n_range;
  int n_blank = 0;
  while (n_blank < p->n_range && p->r_min_m + (n_blank + 0.5) * dr < p->r_blank_m) ++n_blank;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the array keeps the previous call's contents: the maxima must restart at zero
  char* base = reinterpret_cast<char*>(s);
  if (cudaMemsetAsync(base + offsetof(NoAllocScratch, ping_max), 0, sizeof(unsigned int) * n_pings, st) != cudaSuccess)
    return SONAR_E_CUDA;
  const int64_t warps = nb * n_pings;
  k_na_argmax<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(env, n_pings, (int)nb, p->n_range, n_blank, s);
  k_na_compact<<<n_pings, 1024, 0, st>>>(s, pb, p->n_beam_az, p->n_beam_el, p->hfov_rad, p->vfov_rad, p->r_min_m, dr,
                                         p->thr_mode, (float)p->thr, cloud, cloud_cap);
  if (cudaGetLastError() != cudaSuccess) return SONAR_E_CUDA;
  long long counts[kNoAllocMaxPings];
  if (cudaMemcpyAsync(counts, base + offsetof(NoAllocScratch, n_cloud), sizeof(long long) * n_pings,
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SONAR_E_CUDA;
  // as sonar_ping: a count-only call (no cloud buffer) is not a capacity failure
  int rc = SONAR_OK;
  for (int i = 0; i < n_pings; ++i) {
    if (n_cloud) n_cloud[i] = counts[i];
    if (counts[i] > cloud_cap && (cloud_cap > 0 || cloud)) rc = SONAR_E_CAPACITY;
  }
  return rc;
}
