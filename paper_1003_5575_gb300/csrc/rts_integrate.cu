// librtspeel: the visibility integrator (see include/rts_integrate.h).
//
// One CTA per baseline; its threads take the baseline's channels as 16-byte
// halves of a visibility (two polarisations), so every load and store of a
// time sample is coalesced, and sum each group of len consecutive fine
// samples (independent loads, streaming hints); slots past n_fine / len are
// written as zeros.  The kernel streams the cube once: HBM-bound.
#include "rts_integrate.h"
#include "rts_peel.h"

#include <cuda_runtime.h>

#include <cmath>
#include <string>

namespace {

constexpr int kIntThreads = 256;

__global__ void __launch_bounds__(kIntThreads) k_integrate(const float4* __restrict__ fine, float4* __restrict__ out,
                                                           const int* __restrict__ len, int n_fine, int64_t n_bl,
                                                           int n_chan, int n_slot) {
  const int64_t b = blockIdx.x;
  const int L = len[b];
  const int n_out = n_fine / L;
  const float inv = 1.f / (float)L;
  const int n4 = 2 * n_chan;                          // float4 per (time, baseline)
  const size_t tstride = (size_t)n_bl * n4;
  const float4* src = fine + (size_t)b * n4;
  float4* dst = out + (size_t)b * n4;
  for (int i = threadIdx.x; i < n4; i += kIntThreads) {
    for (int s = 0; s < n_slot; ++s) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      if (s < n_out) {
        for (int t = s * L; t < (s + 1) * L; ++t) {
          const float4 x = __ldcs(src + (size_t)t * tstride + i);
          acc.x += x.x; acc.y += x.y; acc.z += x.z; acc.w += x.w;
        }
        acc.x *= inv; acc.y *= inv; acc.z *= inv; acc.w *= inv;
      }
      __stcs(dst + (size_t)s * tstride + i, acc);
    }
  }
}

std::string g_int_init_err;

}  // namespace

struct rts_integ_t {
  int n_fine = 0, n_chan = 0, n_slot = 0;
  int64_t n_bl = 0;
  int device = 0;
  int* d_len = nullptr;
  std::string err;
};

namespace {

int ifail(rts_integ_t* h, int code, const std::string& msg) {
  (h ? h->err : g_int_init_err) = msg;
  return code;
}

}  // namespace

extern "C" {

int rts_integrate_lengths(int32_t n_ant, const double* h_uvw, int32_t n_cut, const double* cut_m,
                          const int32_t* len_for, int32_t* h_len) {
  g_int_init_err.clear();
  if (n_ant < 2 || !h_uvw || !len_for || !h_len) return ifail(nullptr, RTS_EINVAL, "bad arguments");
  if (n_cut < 0 || n_cut > 8 || (n_cut > 0 && !cut_m)) return ifail(nullptr, RTS_EINVAL, "n_cut must be in [0, 8]");
  for (int k = 1; k < n_cut; ++k)
    if (!(cut_m[k] > cut_m[k - 1])) return ifail(nullptr, RTS_EINVAL, "cut_m must be ascending");
  for (int k = 0; k <= n_cut; ++k)
    if (len_for[k] < 1) return ifail(nullptr, RTS_EINVAL, "len_for must be >= 1");
  int64_t bl = 0;
  for (int i = 0; i < n_ant; ++i)
    for (int j = i + 1; j < n_ant; ++j, ++bl) {
      const double du = h_uvw[3 * i] - h_uvw[3 * j], dv = h_uvw[3 * i + 1] - h_uvw[3 * j + 1],
                   dw = h_uvw[3 * i + 2] - h_uvw[3 * j + 2];
      const double d = std::sqrt(du * du + dv * dv + dw * dw);
      int k = 0;
      while (k < n_cut && !(d < cut_m[k])) ++k;
      h_len[bl] = len_for[k];
    }
  return RTS_OK;
}

int rts_integrate_init(int32_t n_fine, int64_t n_bl, int32_t n_chan, const int32_t* h_len, int32_t n_slot,
                       rts_integ_t** out) {
  g_int_init_err.clear();
  if (!out) return ifail(nullptr, RTS_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_fine < 1 || n_fine > 4096) return ifail(nullptr, RTS_EINVAL, "n_fine must be in [1, 4096]");
  if (n_bl < 1 || n_bl >= ((int64_t)1 << 31)) return ifail(nullptr, RTS_EINVAL, "n_bl must be in [1, 2^31 - 1]");
  if (n_chan < 1 || n_chan > 65536) return ifail(nullptr, RTS_EINVAL, "n_chan must be in [1, 65536]");
  if (!h_len) return ifail(nullptr, RTS_EINVAL, "h_len is NULL");
  int min_len = n_fine;
  for (int64_t b = 0; b < n_bl; ++b) {
    if (h_len[b] < 1 || n_fine % h_len[b] != 0)
      return ifail(nullptr, RTS_EINVAL, "every len must be >= 1 and divide n_fine (baseline " + std::to_string(b) + ")");
    if (h_len[b] < min_len) min_len = h_len[b];
  }
  if (n_slot < n_fine / min_len || n_slot > n_fine)
    return ifail(nullptr, RTS_EINVAL, "n_slot must be in [n_fine / min len, n_fine]");
  rts_integ_t* h = new rts_integ_t();
  h->n_fine = n_fine; h->n_bl = n_bl; h->n_chan = n_chan; h->n_slot = n_slot;
  cudaGetDevice(&h->device);
  cudaError_t e = cudaMalloc(&h->d_len, sizeof(int) * (size_t)n_bl);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_len, h_len, sizeof(int) * (size_t)n_bl, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    ifail(nullptr, e == cudaErrorMemoryAllocation ? RTS_ENOMEM : RTS_ECUDA,
          std::string("group lengths: ") + cudaGetErrorString(e));
    rts_integrate_destroy(h);
    return e == cudaErrorMemoryAllocation ? RTS_ENOMEM : RTS_ECUDA;
  }
  *out = h;
  return RTS_OK;
}

int rts_integrate_run(rts_integ_t* h, const void* d_fine, void* d_out, void* stream) {
  if (!h) return ifail(nullptr, RTS_EINVAL, "handle is NULL");
  if (!d_fine || !d_out) return ifail(h, RTS_EINVAL, "d_fine and d_out are required");
  if ((reinterpret_cast<uintptr_t>(d_fine) | reinterpret_cast<uintptr_t>(d_out)) & 15u)
    return ifail(h, RTS_EINVAL, "d_fine and d_out must start on a 16-byte boundary");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_integrate<<<(unsigned)h->n_bl, kIntThreads, 0, s>>>(static_cast<const float4*>(d_fine), static_cast<float4*>(d_out),
                                                        h->d_len, h->n_fine, h->n_bl, h->n_chan, h->n_slot);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ifail(h, RTS_ECUDA, std::string("integrator launch: ") + cudaGetErrorString(e));
  return RTS_OK;
}

const char* rts_integrate_last_error(const rts_integ_t* h) { return h ? h->err.c_str() : g_int_init_err.c_str(); }

void rts_integrate_destroy(rts_integ_t* h) {
  if (!h) return;
  int prev = -1;
  if (cudaGetDevice(&prev) == cudaSuccess && prev != h->device) cudaSetDevice(h->device);
  if (h->d_len) cudaFree(h->d_len);
  if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
  delete h;
}

}  // extern "C"
