// Deterministic exclusive prefix scan (int32 counts -> int64 offsets), used for
// the two-pass CSR build (row counts -> row_ptr), active-point compaction and
// the radix-sort digit offsets.  Three phases: per-block sums, one-block scan
// of the block sums, per-block re-scan with the block offset.
#include "gp_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = gp::kScanItems / kThreads;  // 16 contiguous items per thread

__device__ inline long long warp_incl_scan(long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; every thread gets
// its exclusive prefix as the return value and the block total in *total.
__device__ inline long long block_excl_scan(long long v, long long* total) {
  __shared__ long long warp_tot[kThreads / 32];
  __shared__ long long block_total;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    long long t = lane < kThreads / 32 ? warp_tot[lane] : 0;
    long long ti = warp_incl_scan(t);
    if (lane < kThreads / 32) warp_tot[lane] = ti - t;
    if (lane == kThreads / 32 - 1) block_total = ti;
  }
  __syncthreads();
  long long r = inc - v + warp_tot[w];
  *total = block_total;
  __syncthreads();  // the shared words may be reused by the next call
  return r;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int32_t* __restrict__ in, int64_t n,
                                                          int64_t* __restrict__ part) {
  const int64_t base = (int64_t)blockIdx.x * gp::kScanItems + (int64_t)threadIdx.x * kPerThread;
  long long s = 0;
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    int64_t idx = base + i;
    if (idx < n) s += in[idx];
  }
  long long tot = 0;
  (void)block_excl_scan(s, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// One block: exclusive scan of nparts block sums in place; part[nparts] = total.
__global__ void __launch_bounds__(kThreads) k_scan_parts(int64_t* part, int nparts) {
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nparts; base += kThreads) {
    int i = base + threadIdx.x;
    long long v = i < nparts ? part[i] : 0;
    long long tot = 0;
    long long ex = block_excl_scan(v, &tot);
    if (i < nparts) part[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) part[nparts] = carry;
}

__global__ void __launch_bounds__(kThreads) k_scan_down(const int32_t* __restrict__ in, int64_t n,
                                                        const int64_t* __restrict__ part,
                                                        int64_t* __restrict__ out, int nparts) {
  const int64_t base = (int64_t)blockIdx.x * gp::kScanItems + (int64_t)threadIdx.x * kPerThread;
  int32_t v[kPerThread];
  long long s = 0;
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    int64_t idx = base + i;
    v[i] = idx < n ? in[idx] : 0;
    s += v[i];
  }
  long long tot = 0;
  long long ex = block_excl_scan(s, &tot) + part[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = ex;
    ex += v[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = part[nparts];
}

}  // namespace

namespace gp {

int scan_i32_to_i64(gp_ctx* c, const int32_t* in, int64_t* out, int64_t n) {
  if (n == 0) {
    GP_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), c->stream));
    return GP_OK;
  }
  const int64_t nparts = (n + kScanItems - 1) / kScanItems;
  if (nparts > (int64_t)1 << 30) return GP_ERR_UNSUPPORTED;
  GP_CHECK(ensure(c, c->scan_part, (size_t)(nparts + 1) * sizeof(int64_t)));
  int64_t* part = (int64_t*)c->scan_part.p;
  k_scan_reduce<<<(unsigned)nparts, kThreads, 0, c->stream>>>(in, n, part);
  GP_LAUNCH_CHECK();
  k_scan_parts<<<1, kThreads, 0, c->stream>>>(part, (int)nparts);
  GP_LAUNCH_CHECK();
  k_scan_down<<<(unsigned)nparts, kThreads, 0, c->stream>>>(in, n, part, out, (int)nparts);
  GP_LAUNCH_CHECK();
  c->launches += 3;
  return GP_OK;
}

}  // namespace gp
