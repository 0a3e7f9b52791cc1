// gp_get_csr_noalloc: the copy-out of gp_get_csr with its only scratch buffer
// (the unscaled values, staged on the device before the copy to the caller)
// in static device memory, so the call allocates nothing.  For callers that
// must not allocate device memory at this point (another allocator owns the
// device's memory, or the process is at its device-memory limit).
#include <mutex>

#include "gp_internal.cuh"

namespace {

// Staging area shared by every call on a device.  In host code the name is
// only a host-side handle; kernels receive the device address looked up once
// per device with cudaGetSymbolAddress.
static __device__ __align__(256) double g_stage[GP_NOALLOC_MAX_NNZ];

constexpr int kMaxDevices = 64;
double* g_stage_addr[kMaxDevices] = {};
std::mutex g_stage_mu;

// Device address of g_stage on `device` (which must be current).
int stage_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return GP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_stage_mu);
  if (!g_stage_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_stage);
    if (e != cudaSuccess) return gp::cuda_status(e);
    g_stage_addr[device] = (double*)p;
  }
  *out = g_stage_addr[device];
  return GP_OK;
}

// Same arithmetic as the unscaling in gp_get_csr: K = D^1/2 Khat D^1/2.
template <typename T>
__global__ void __launch_bounds__(256) k_unscale_to_stage(int64_t n, const int64_t* __restrict__ rp,
                                                          const int32_t* __restrict__ col,
                                                          const T* __restrict__ val,
                                                          const double* __restrict__ dinv64,
                                                          double* __restrict__ stage) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t p = (int64_t)blockIdx.x * 8 + w; p < n; p += (int64_t)gridDim.x * 8) {
    const double dp = dinv64[p];
    for (int64_t e = rp[p] + lane; e < rp[p + 1]; e += 32) stage[e] = (double)val[e] / (dp * dinv64[col[e]]);
  }
}

int copy_to(gp_ctx* c, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return GP_OK;
  GP_CUDA(cudaMemcpyAsync(dst, src, bytes,
                          gp::is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  return GP_OK;
}

}  // namespace

extern "C" int gp_get_csr_noalloc(gp_ctx* c, int64_t* row_ptr, int32_t* col, double* val, int32_t* perm,
                                  int64_t sizes[2]) {
  if (!c || !sizes) return GP_ERR_INVALID_ARG;
  if (!c->assembled) return GP_ERR_NOT_ASSEMBLED;
  GP_CUDA(cudaSetDevice(c->device));
  sizes[0] = c->n_act;
  sizes[1] = c->nnz;
  if (val && c->nnz > (int64_t)GP_NOALLOC_MAX_NNZ) return GP_ERR_UNSUPPORTED;
  if (c->n_act == 0) {
    if (row_ptr) {
      const int64_t z = 0;
      if (gp::is_device_ptr(row_ptr)) {
        GP_CUDA(cudaMemcpyAsync(row_ptr, &z, sizeof(z), cudaMemcpyHostToDevice, c->stream));
        GP_CUDA(cudaStreamSynchronize(c->stream));
      } else {
        *row_ptr = 0;
      }
    }
    return GP_OK;
  }
  if (row_ptr) GP_CHECK(copy_to(c, row_ptr, c->row_ptr.p, (size_t)(c->n_act + 1) * sizeof(int64_t)));
  if (col) GP_CHECK(copy_to(c, col, c->col.p, (size_t)c->nnz * sizeof(int32_t)));
  if (perm) GP_CHECK(copy_to(c, perm, c->vals.p, (size_t)c->n_act * sizeof(int32_t)));
  if (val) {
    double* stage = nullptr;
    GP_CHECK(stage_address(c->device, &stage));
    int64_t blocks = (c->n_act + 7) / 8;
    if (blocks > (int64_t)c->num_sms * 8) blocks = (int64_t)c->num_sms * 8;
    if (c->precision == GP_FP64)
      k_unscale_to_stage<double><<<(unsigned)blocks, 256, 0, c->stream>>>(
          c->n_act, (const int64_t*)c->row_ptr.p, (const int32_t*)c->col.p, (const double*)c->val.p,
          (const double*)c->dinv64.p, stage);
    else
      k_unscale_to_stage<float><<<(unsigned)blocks, 256, 0, c->stream>>>(
          c->n_act, (const int64_t*)c->row_ptr.p, (const int32_t*)c->col.p, (const float*)c->val.p,
          (const double*)c->dinv64.p, stage);
    GP_LAUNCH_CHECK();
    GP_CHECK(copy_to(c, val, stage, (size_t)c->nnz * sizeof(double)));
  }
  GP_CUDA(cudaStreamSynchronize(c->stream));
  return GP_OK;
}
