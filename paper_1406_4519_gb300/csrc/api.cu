// api.cu -- the C ABI of libdfacto (include/dfacto.h): argument checks, handle
// lifetime, factor conversion, and the ALS / GD / fit drivers.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "device.cuh"
#include "internal.h"
#include "smem_optin.h"

namespace dfacto {

std::atomic<long long> g_launches{0};

cudaError_t ensure_dynamic_smem(const void* kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static SmemOptIn optin;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  return static_cast<cudaError_t>(optin.ensure(kernel, dev, bytes, [&] {
    return static_cast<int>(
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  }));
}

dfacto_status fail(dfacto_t* h, dfacto_status s, const std::string& what) {
  if (h) h->err = what;
  return s;
}

dfacto_status cuda_fail(dfacto_t* h, cudaError_t e, const char* what) {
  if (h) h->err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a non-sticky error
  return e == cudaErrorMemoryAllocation ? DFACTO_ENOMEM : DFACTO_ECUDA;
}

// Device memory of a handle comes from the device's stream-ordered pool
// (cudaMallocAsync on the handle's stream): allocation and release do not
// synchronize the device, so building and destroying many small handles (a
// serving loop) does not stall the work of others.  Freed memory stays cached
// in the pool for the next handle (release threshold raised once per device).
void keep_pool_memory() {
  static std::once_flag once[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  std::call_once(once[dev], [dev]() {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  });
}

dfacto_status dalloc(dfacto_t* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(p, bytes, h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(h, e == cudaErrorMemoryAllocation ? DFACTO_ENOMEM : DFACTO_ECUDA,
                std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  h->bytes += (int64_t)bytes;
  return DFACTO_OK;
}

void dfree(dfacto_t* h, void* p, size_t bytes) {
  if (!p) return;
  cudaFreeAsync(p, h->stream);
  if (bytes == 0) bytes = 16;
  h->bytes -= (int64_t)bytes;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

namespace {

size_t elem_size(int dtype) {
  return dtype == DFACTO_BF16 ? 2 : (dtype == DFACTO_F64 ? 8 : 4);
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    if constexpr (std::is_same<D, __nv_bfloat16>::value) {
      if constexpr (std::is_same<S, double>::value) dst[t] = __double2bfloat16(src[t]);
      else if constexpr (std::is_same<S, __nv_bfloat16>::value) dst[t] = src[t];
      else dst[t] = __float2bfloat16_rn((float)src[t]);
    } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
      dst[t] = (D)__bfloat162float(src[t]);
    } else {
      dst[t] = (D)src[t];
    }
  }
}

template <typename S>
cudaError_t convert_from(const S* src, void* dst, int dst_dtype, int64_t n, cudaStream_t s) {
  const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
  if (dst_dtype == DFACTO_F32) {
    convert_kernel<S, float><<<nb, 256, 0, s>>>(src, (float*)dst, n);
  } else if (dst_dtype == DFACTO_BF16) {
    convert_kernel<S, __nv_bfloat16><<<nb, 256, 0, s>>>(src, (__nv_bfloat16*)dst, n);
  } else {
    convert_kernel<S, double><<<nb, 256, 0, s>>>(src, (double*)dst, n);
  }
  DF_COUNT();
  return cudaGetLastError();
}

cudaError_t convert(const void* src, int src_dtype, void* dst, int dst_dtype, int64_t n,
                    cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (src_dtype == DFACTO_F32) return convert_from((const float*)src, dst, dst_dtype, n, s);
  if (src_dtype == DFACTO_BF16) return convert_from((const __nv_bfloat16*)src, dst, dst_dtype, n, s);
  return convert_from((const double*)src, dst, dst_dtype, n, s);
}

__global__ void fill_double(double* p, int n, double v) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = v;
}

dfacto_status read_back(dfacto_t* h) {
  DF_CUDA(h, cudaMemcpyAsync(h->host_scal, h->scal, sizeof(double) * kNumScalars,
                             cudaMemcpyDeviceToHost, h->stream));
  DF_CUDA(h, cudaMemcpyAsync(h->host_flags, h->flags, sizeof(int32_t) * kNumFlags,
                             cudaMemcpyDeviceToHost, h->stream));
  DF_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->host_flags[kFlagInternal]) return fail(h, DFACTO_EINTERNAL, "internal consistency check failed");
  return DFACTO_OK;
}

bool valid_mode(int mode) { return mode >= 0 && mode < 3; }

}  // namespace

dfacto_status grow_partials(dfacto_t* h, int64_t n) {
  if (n <= h->partials_cap) return DFACTO_OK;
  dfree(h, h->partials, sizeof(double) * (size_t)h->partials_cap);
  h->partials = nullptr;
  h->partials_cap = 0;
  dfacto_status st = dalloc(h, reinterpret_cast<void**>(&h->partials), sizeof(double) * (size_t)n);
  if (st == DFACTO_OK) h->partials_cap = n;
  return st;
}

dfacto_status convert_factor_in(dfacto_t* h, int m, const void* src, int src_dtype) {
  const int64_t n = (int64_t)h->dims[m] * h->R;
  const void* dsrc = src;
  void* tmp = nullptr;
  if (!is_device_ptr(src) && src_dtype == h->dtype) {  // same type: one copy into the factor
    DF_CUDA(h, cudaMemcpyAsync(h->F[m], src, n * elem_size(src_dtype), cudaMemcpyHostToDevice, h->stream));
    DF_CUDA(h, cudaStreamSynchronize(h->stream));  // caller may free its host buffer
    h->gram_valid[m] = false;
    return DFACTO_OK;
  }
  if (!is_device_ptr(src)) {
    DF_CUDA(h, cudaMallocAsync(&tmp, std::max<size_t>(16, n * elem_size(src_dtype)), h->stream));
    DF_CUDA(h, cudaMemcpyAsync(tmp, src, n * elem_size(src_dtype), cudaMemcpyHostToDevice, h->stream));
    dsrc = tmp;
  }
  cudaError_t e = convert(dsrc, src_dtype, h->F[m], h->dtype, n, h->stream);
  if (tmp) cudaFreeAsync(tmp, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "factor conversion");
  if (tmp) DF_CUDA(h, cudaStreamSynchronize(h->stream));  // caller may free its host buffer
  h->gram_valid[m] = false;
  return DFACTO_OK;
}

dfacto_status convert_factor_out(dfacto_t* h, int m, void* dst, int dst_dtype) {
  const int64_t n = (int64_t)h->dims[m] * h->R;
  if (is_device_ptr(dst)) {
    cudaError_t e = convert(h->F[m], h->dtype, dst, dst_dtype, n, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "factor conversion");
    return DFACTO_OK;
  }
  if (dst_dtype == h->dtype) {  // same type: one copy out of the factor
    DF_CUDA(h, cudaMemcpyAsync(dst, h->F[m], n * elem_size(dst_dtype), cudaMemcpyDeviceToHost, h->stream));
    DF_CUDA(h, cudaStreamSynchronize(h->stream));
    return DFACTO_OK;
  }
  void* tmp = nullptr;
  DF_CUDA(h, cudaMallocAsync(&tmp, std::max<size_t>(16, n * elem_size(dst_dtype)), h->stream));
  cudaError_t e = convert(h->F[m], h->dtype, tmp, dst_dtype, n, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst, tmp, n * elem_size(dst_dtype), cudaMemcpyDeviceToHost, h->stream);
  cudaFreeAsync(tmp, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "factor read-back");
  DF_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFACTO_OK;
}

}  // namespace dfacto

using namespace dfacto;

extern "C" {

void dfacto_options_init(dfacto_options* opt, int32_t rank) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->rank = rank;
  opt->factor_dtype = DFACTO_F32;
  opt->lambda_reg = 0.0;
}

const char* dfacto_status_str(dfacto_status s) {
  switch (s) {
    case DFACTO_OK: return "ok";
    case DFACTO_EINVAL: return "invalid argument";
    case DFACTO_ERANGE: return "coordinate out of range";
    case DFACTO_EDUP: return "duplicate coordinate";
    case DFACTO_ENOMEM: return "out of memory";
    case DFACTO_ECUDA: return "CUDA error";
    case DFACTO_ESINGULAR: return "singular Gram-Hadamard matrix (pseudo-inverse used)";
    case DFACTO_ELSFAIL: return "line search failed";
    case DFACTO_ETIMEOUT: return "device wait timed out";
    case DFACTO_EINTERNAL: return "internal error";
  }
  return "unknown status";
}

void dfacto_destroy(dfacto_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  joint_free(h);
  if (h->batch) {  // the factors belong to the batch's pools
    batch_forget(h->batch, h);
    for (int m = 0; m < 3; ++m) h->F[m] = nullptr;
  }
  for (int m = 0; m < 3; ++m) {
    ModeCSR& M = h->m[m];
    for (void* q : {(void*)M.fiber_ptr, (void*)M.fiber_idx, (void*)M.fiber_row, (void*)M.nz_ptr,
                    (void*)M.nz_idx, (void*)M.nz_val, (void*)M.end_bits, (void*)M.seg_fib,
                    h->F[m], (void*)h->grad[m], (void*)h->gram[m]})
      if (q) cudaFreeAsync(q, h->stream);
  }
  for (void* q : {(void*)h->N, (void*)h->Fh, (void*)h->lambda, (void*)h->inv_lambda, (void*)h->ipart,
                  (void*)h->gd_mats, (void*)h->gd_scratch, (void*)h->W, (void*)h->rr_work, (void*)h->W32, (void*)h->scal,
                  (void*)h->flags, (void*)h->partials, (void*)h->carry, (void*)h->carry_row,
                  (void*)h->pad_in, (void*)h->pad_f, (void*)h->pad_out, (void*)h->pad_dual,
                  (void*)h->ls_vals})
    if (q) cudaFreeAsync(q, h->stream);
  delete[] h->host_scal;
  delete[] h->host_flags;
  if (h->aux) {
    cudaStreamSynchronize(h->aux);
    cudaStreamDestroy(h->aux);
  }
  if (h->aux_fork) cudaEventDestroy(h->aux_fork);
  if (h->aux_join) cudaEventDestroy(h->aux_join);
  cudaGetLastError();
  delete h;
}

const char* dfacto_last_error(const dfacto_t* h) { return h ? h->err.c_str() : ""; }

int64_t dfacto_launch_count(void) { return (int64_t)g_launches.load(); }

dfacto_status dfacto_build(const int32_t* idx, const float* val, int64_t nnz, const int32_t dims[3],
                           const dfacto_options* opt_in, void* stream, dfacto_t** out) {
  if (!out) return DFACTO_EINVAL;
  *out = nullptr;
  if (!dims || nnz < 0 || nnz > kMaxNnz || (nnz > 0 && (!idx || !val)))
    return DFACTO_EINVAL;
  for (int m = 0; m < 3; ++m)
    if (dims[m] < 1) return DFACTO_EINVAL;
  dfacto_options opt;
  if (opt_in) opt = *opt_in;
  else dfacto_options_init(&opt, 1);
  const int R = opt.rank;
  if (R < 1 || R > 128 || (R > 32 && R % 4 != 0)) return DFACTO_EINVAL;
  if (opt.factor_dtype != DFACTO_F32 && opt.factor_dtype != DFACTO_BF16) return DFACTO_EINVAL;
  if (!(opt.lambda_reg >= 0.0)) return DFACTO_EINVAL;
  if (opt.vec != 0 && (opt.vec != 1 && opt.vec != 2 && opt.vec != 4 && opt.vec != 8)) return DFACTO_EINVAL;
  if (opt.vec != 0 && R % opt.vec != 0) return DFACTO_EINVAL;
  if (opt.seg_nnz < 0 || opt.seg_nnz > kMaxSeg) return DFACTO_EINVAL;
  if (opt.walk < 0 || opt.walk > 2) return DFACTO_EINVAL;
  if (opt.line_search != 0 && opt.line_search != 1) return DFACTO_EINVAL;

  dfacto_t* h = new (std::nothrow) dfacto_handle();
  if (!h) return DFACTO_ENOMEM;
  keep_pool_memory();
  h->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&h->device);
  std::memcpy(h->dims, dims, sizeof(int32_t) * 3);
  h->nnz = nnz;
  h->R = R;
  h->dtype = opt.factor_dtype;
  h->lambda_reg = opt.lambda_reg;
  h->opt = opt;
  auto bail = [&](dfacto_status st) {
    dfacto_destroy(h);
    return st;
  };
  dfacto_status st = DFACTO_OK;
  const size_t RR = (size_t)R * R;
  const int64_t maxdim = std::max<int64_t>(dims[0], std::max<int64_t>(dims[1], dims[2]));
  if ((st = dalloc(h, (void**)&h->scal, sizeof(double) * kNumScalars)) != DFACTO_OK) return bail(st);
  if ((st = dalloc(h, (void**)&h->flags, sizeof(int32_t) * kNumFlags)) != DFACTO_OK) return bail(st);
  if ((st = grow_partials(h, std::max<int64_t>(608 * (int64_t)RR, 4096))) != DFACTO_OK) return bail(st);
  if ((st = dalloc(h, (void**)&h->lambda, sizeof(double) * R)) != DFACTO_OK) return bail(st);
  if ((st = dalloc(h, (void**)&h->inv_lambda, sizeof(float) * R)) != DFACTO_OK) return bail(st);
  if ((st = dalloc(h, (void**)&h->ipart, sizeof(double) * 608 * R)) != DFACTO_OK) return bail(st);  // >= blocks
  if ((st = dalloc(h, (void**)&h->gd_mats, sizeof(double) * 9 * RR)) != DFACTO_OK) return bail(st);
  if ((st = dalloc(h, (void**)&h->gd_scratch, sizeof(uint32_t) * 8)) != DFACTO_OK) return bail(st);
  if ((st = dalloc(h, (void**)&h->W, sizeof(double) * RR)) != DFACTO_OK) return bail(st);
  if ((st = dalloc(h, (void**)&h->rr_work, sizeof(double) * (2 * RR + R))) != DFACTO_OK) return bail(st);
  if ((st = dalloc(h, (void**)&h->W32, sizeof(float) * RR)) != DFACTO_OK) return bail(st);
  if ((st = dalloc(h, (void**)&h->N, sizeof(float) * maxdim * R)) != DFACTO_OK) return bail(st);
  if (R > 32 && (st = dalloc(h, (void**)&h->Fh, sizeof(float) * maxdim * R)) != DFACTO_OK)
    return bail(st);  // N Gamma^{-1} is stored only by the row passes for R > 32
  for (int m = 0; m < 3; ++m) {
    if ((st = dalloc(h, &h->F[m], elem_size(h->dtype) * (size_t)dims[m] * R)) != DFACTO_OK) return bail(st);
    if ((st = dalloc(h, (void**)&h->gram[m], sizeof(double) * RR)) != DFACTO_OK) return bail(st);
  }
  if (cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->aux_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->aux_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return bail(DFACTO_ECUDA);
  }
  h->host_scal = new (std::nothrow) double[kNumScalars]();
  h->host_flags = new (std::nothrow) int32_t[kNumFlags]();
  if (!h->host_scal || !h->host_flags) return bail(DFACTO_ENOMEM);
  cudaStream_t s = h->stream;
  if (cudaMemsetAsync(h->scal, 0, sizeof(double) * kNumScalars, s) != cudaSuccess) return bail(DFACTO_ECUDA);
  for (int m = 0; m < 3; ++m)
    if (cudaMemsetAsync(h->F[m], 0, elem_size(h->dtype) * (size_t)dims[m] * R, s) != cudaSuccess)
      return bail(DFACTO_ECUDA);
  fill_double<<<1, 128, 0, s>>>(h->lambda, R, 1.0); DF_COUNT();

  // COO on the device.
  const int32_t* d_idx = idx;
  const float* d_val = val;
  int32_t* tmp_idx = nullptr;
  float* tmp_val = nullptr;
  if (nnz > 0 && !is_device_ptr(idx)) {
    if (cudaMallocAsync((void**)&tmp_idx, sizeof(int32_t) * 3 * nnz, s) != cudaSuccess ||
        cudaMemcpyAsync(tmp_idx, idx, sizeof(int32_t) * 3 * nnz, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      return bail(DFACTO_ENOMEM);
    }
    d_idx = tmp_idx;
  }
  if (nnz > 0 && !is_device_ptr(val)) {
    if (cudaMallocAsync((void**)&tmp_val, sizeof(float) * nnz, s) != cudaSuccess ||
        cudaMemcpyAsync(tmp_val, val, sizeof(float) * nnz, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      if (tmp_idx) cudaFreeAsync(tmp_idx, s);
      return bail(DFACTO_ENOMEM);
    }
    d_val = tmp_val;
  }
  st = build_modes(h, d_idx, d_val);
  if (tmp_idx) cudaFreeAsync(tmp_idx, s);
  if (tmp_val) cudaFreeAsync(tmp_val, s);
  if (st != DFACTO_OK) {
    const std::string msg = h->err;
    dfacto_destroy(h);
    (void)msg;
    return st;
  }
  for (int m = 0; m < 3; ++m) {
    h->m[m].cfg = choose_walk(R, h->dtype, nnz, h->m[m].nfib, opt.seg_nnz, opt.vec);
    if (opt.walk > 0) {
      h->m[m].cfg.kernel = opt.walk;
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return bail(DFACTO_ECUDA);
  *out = h;
  return DFACTO_OK;
}

dfacto_status dfacto_get_info(dfacto_t* h, dfacto_info* info) {
  if (!h || !info) return DFACTO_EINVAL;
  std::memset(info, 0, sizeof(*info));
  std::memcpy(info->dims, h->dims, sizeof(h->dims));
  info->rank = h->R;
  info->nnz = h->nnz;
  const int RP = walk_rank(h->R, h->opt.vec);
  for (int m = 0; m < 3; ++m) {
    info->nfib[m] = h->m[m].nfib;
    info->seg_nnz[m] = h->m[m].cfg.seg;
    info->vec[m] = (RP != h->R)
                       ? choose_walk(RP, DFACTO_F32, h->nnz, h->m[m].nfib, h->opt.seg_nnz, 0).vec
                       : h->m[m].cfg.vec;
  }
  info->device_bytes = h->bytes;
  info->factor_dtype = h->dtype;
  double nx2 = 0.0;
  DF_CUDA(h, cudaMemcpyAsync(&nx2, h->scal + kNormX2, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  DF_CUDA(h, cudaStreamSynchronize(h->stream));
  info->norm_x2 = nx2;
  return DFACTO_OK;
}

dfacto_status dfacto_set_stream(dfacto_t* h, void* stream) {
  if (!h) return DFACTO_EINVAL;
  h->stream = static_cast<cudaStream_t>(stream);
  return DFACTO_OK;
}

dfacto_status dfacto_sync(dfacto_t* h) {
  if (!h) return DFACTO_EINVAL;
  DF_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFACTO_OK;
}

dfacto_status dfacto_set_factors(dfacto_t* h, int mode, const void* F, dfacto_dtype dtype) {
  if (!h || !valid_mode(mode) || !F) return DFACTO_EINVAL;
  if (dtype != DFACTO_F32 && dtype != DFACTO_BF16 && dtype != DFACTO_F64) return DFACTO_EINVAL;
  return convert_factor_in(h, mode, F, dtype);
}

dfacto_status dfacto_get_factors(dfacto_t* h, int mode, void* F, dfacto_dtype dtype) {
  if (!h || !valid_mode(mode) || !F) return DFACTO_EINVAL;
  if (dtype != DFACTO_F32 && dtype != DFACTO_BF16 && dtype != DFACTO_F64) return DFACTO_EINVAL;
  return convert_factor_out(h, mode, F, dtype);
}

dfacto_status dfacto_get_lambda(dfacto_t* h, double* lambda) {
  if (!h || !lambda) return DFACTO_EINVAL;
  DF_CUDA(h, cudaMemcpyAsync(lambda, h->lambda, sizeof(double) * h->R, cudaMemcpyDeviceToHost, h->stream));
  DF_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFACTO_OK;
}

dfacto_status dfacto_set_lambda(dfacto_t* h, const double* lambda) {
  if (!h || !lambda) return DFACTO_EINVAL;
  DF_CUDA(h, cudaMemcpyAsync(h->lambda, lambda, sizeof(double) * h->R, cudaMemcpyHostToDevice, h->stream));
  DF_CUDA(h, cudaStreamSynchronize(h->stream));
  return DFACTO_OK;
}

dfacto_status dfacto_mttkrp(dfacto_t* h, int mode, float* out) {
  if (!h || !valid_mode(mode) || !out) return DFACTO_EINVAL;
  if (!is_device_ptr(out)) return fail(h, DFACTO_EINVAL, "dfacto_mttkrp: out must be device memory");
  return mttkrp_launch(h, mode, out);
}

dfacto_status dfacto_als_iter(dfacto_t* h, double* fit_out) {
  if (!h) return DFACTO_EINVAL;
  DF_CUDA(h, cudaMemsetAsync(h->flags, 0, sizeof(int32_t) * kNumFlags, h->stream));
  dfacto_status st;
  for (int mode = 0; mode < 3; ++mode)
    if ((st = als_mode(h, mode)) != DFACTO_OK) return st;
  if ((st = als_fit(h)) != DFACTO_OK) return st;
  if (!fit_out) return DFACTO_OK;
  if ((st = read_back(h)) != DFACTO_OK) return st;
  *fit_out = h->host_scal[kFit];
  return h->host_flags[kFlagSingular] ? DFACTO_ESINGULAR : DFACTO_OK;
}

dfacto_status dfacto_gd_iter(dfacto_t* h, double* loss_out, double* alpha_out) {
  if (!h) return DFACTO_EINVAL;
  dfacto_status st;
  for (int m = 0; m < 3; ++m)
    if (!h->grad[m] &&
        (st = dalloc(h, (void**)&h->grad[m], sizeof(float) * (size_t)h->dims[m] * h->R)) != DFACTO_OK)
      return st;
  DF_CUDA(h, cudaMemsetAsync(h->flags, 0, sizeof(int32_t) * kNumFlags, h->stream));
  if ((st = gd_step(h)) != DFACTO_OK) return st;
  if (!loss_out && !alpha_out) return DFACTO_OK;
  if ((st = read_back(h)) != DFACTO_OK) return st;
  if (loss_out) *loss_out = h->host_scal[kLoss];
  if (alpha_out) *alpha_out = h->host_scal[kStep];
  return h->host_flags[kFlagLsFail] ? DFACTO_ELSFAIL : DFACTO_OK;
}

dfacto_status dfacto_fit(dfacto_t* h, double* fit_out) {
  if (!h || !fit_out) return DFACTO_EINVAL;
  DF_CUDA(h, cudaMemsetAsync(h->flags, 0, sizeof(int32_t) * kNumFlags, h->stream));
  dfacto_status st = fit_direct(h);
  if (st != DFACTO_OK) return st;
  if ((st = read_back(h)) != DFACTO_OK) return st;
  *fit_out = h->host_scal[kFit];
  return DFACTO_OK;
}

dfacto_status dfacto_get_csr(dfacto_t* h, int mode, dfacto_csr_view* v) {
  if (!h || !valid_mode(mode) || !v) return DFACTO_EINVAL;
  const ModeCSR& M = h->m[mode];
  v->dim_o = M.dim_o;
  v->nfib = M.nfib;
  v->nnz = h->nnz;
  v->fiber_ptr = M.fiber_ptr;
  v->fiber_idx = M.fiber_idx;
  v->nz_ptr = M.nz_ptr;
  v->nz_idx = M.nz_idx;
  v->nz_val = M.nz_val;
  return DFACTO_OK;
}

}  // extern "C"
