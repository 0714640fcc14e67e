// ctof_forward_static: the forward operator m = A mu with every intermediate
// held in a fixed, file-scope device array instead of memory allocated by the
// library.
//
// Who needs this: callers that may not allocate device memory at the point of
// the call -- real-time acquisition loops that must never wait on an
// allocator (cudaMalloc/cudaFree can synchronise the device), and host
// frameworks or plugins that own every device allocation themselves and hand
// the library only input and output buffers.  This entry point performs no
// cudaMalloc, cudaFree or other allocating call; the caller passes the handle
// (built beforehand), the input volume and the output buffer.
//
// The scratch array (CTOF_STATIC_SCRATCH_BYTES, 32 MiB) is part of the loaded
// library image: every GPU that loads the library holds it until the process
// exits.  All calls share it, so calls that overlap on the GPU (different
// streams, or several handles at once) race on it and corrupt each other's
// results; serialise them.  Every scratch byte that is read is written earlier
// in the same call, so nothing has to start at zero.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "ctof_internal.h"

#define CTOF_STATIC_SCRATCH_BYTES (32u << 20)
#define CTOF_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_forward_scratch[CTOF_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_setup_mutex;
void* g_scratch_ptr[CTOF_MAX_DEVICES] = {};

// Device address of the scratch array on `dev`, resolved once per device with
// that device current (the host-side symbol is only a stand-in) and kept for
// the life of the process: the first call on a device does this set-up, so it
// must come before any stream capture.  A cudaDeviceReset destroys the
// context the address belongs to; the kept address is then stale, and the
// entry point must not be called again in that process.
ctof_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= CTOF_MAX_DEVICES) return CTOF_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    CTOF_CUDA_TRY(cudaGetSymbolAddress(&p, g_forward_scratch));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return CTOF_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" ctof_status ctof_forward_static(ctof_kernel k, const float* d_mu, float* d_m, void* stream) {
  if (!k || !d_mu || !d_m) return CTOF_EINVAL;
  // scratch: Z-side row spectra, Z-side spectrum, T-side spectrum, T-side row spectra
  const size_t b_iz = align256(fft_inter_elems(k, k->nz, k->n) * sizeof(float2));
  const size_t b_sz = align256((size_t)k->nf * k->ldz * sizeof(float2));
  const size_t b_st = align256((size_t)k->nf * k->ldt * sizeof(float2));
  const size_t b_it = align256(fft_inter_elems(k, k->nt, k->n) * sizeof(float2));
  const size_t need = b_iz + b_sz + b_st + b_it;
  if (need > CTOF_STATIC_SCRATCH_BYTES) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "ctof_forward_static: this grid needs %zu bytes of scratch, the static maximum is %u bytes", need,
             (unsigned)CTOF_STATIC_SCRATCH_BYTES);
    ctof_set_last_error_text(msg);
    return CTOF_EUNSUPPORTED;
  }
  int prev = -1;
  CTOF_CUDA_TRY(cudaGetDevice(&prev));
  if (prev != k->device) CTOF_CUDA_TRY(cudaSetDevice(k->device));
  void* base = nullptr;
  ctof_status s = scratch_address(k->device, &base);
  if (s == CTOF_OK) {
    char* p = static_cast<char*>(base);
    float2* inter_z = reinterpret_cast<float2*>(p);
    float2* spec_z = reinterpret_cast<float2*>(p + b_iz);
    float2* spec_t = reinterpret_cast<float2*>(p + b_iz + b_sz);
    float2* inter_t = reinterpret_cast<float2*>(p + b_iz + b_sz + b_st);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = fft_forward_planes(k, d_mu, k->nz, k->n, k->n, k->n, inter_z, spec_z, k->ldz, st);
    if (s == CTOF_OK) s = contract_forward(k, spec_z, spec_t, st);
    if (s == CTOF_OK) s = fft_inverse_planes(k, spec_t, k->ldt, k->nt, k->n, k->n, inter_t, d_m, k->n, st);
  }
  if (prev != k->device) cudaSetDevice(prev);
  return s;
}
