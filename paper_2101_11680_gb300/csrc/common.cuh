// Shared device/host helpers of the ctof library (complex arithmetic, error
// plumbing).  Internal header: not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ctof.h"

#define CTOF_CUDA_TRY(expr)                                  \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) {                                 \
      ctof_set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return CTOF_ECUDA;                                     \
    }                                                        \
  } while (0)

#define CTOF_TRY(expr)              \
  do {                              \
    ctof_status _s = (expr);        \
    if (_s != CTOF_OK) return _s;   \
  } while (0)

void ctof_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void ctof_set_last_error_text(const char* msg);

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

static inline int ctof_round_up(int x, int m) { return (x + m - 1) / m * m; }
static inline int ctof_div_up(long long x, long long m) { return (int)((x + m - 1) / m); }
