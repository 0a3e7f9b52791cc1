// The randomized log-determinant the paper cites (Sec. 2.5: Boutsidis et al.),
// as an alternative to stochastic Lanczos quadrature on the same split
//   ln|K| = sum_act ln D + ln|Khat| + N_inact ln sigma_n^2.
// With a >= lambda_max(Khat) and C = I - Khat / a,
//   ln|Khat| = N_act ln a + ln|I - C| = N_act ln a - sum_{k>=1} tr(C^k) / k,
// truncated after m terms, each trace taken as z^T C^k z for the same
// Rademacher probes the solves use:
//   Gamma_l = N_act ln a - sum_{k=1}^{m} z_l^T C^k z_l / k.
// a is the Gershgorin bound max_i sum_j |Khat_ij| of the stored FP32 matrix
// (any a >= lambda_max is valid; the cited method estimates it by power
// iterations instead).  V_k = C^k Z is one batched SpMM (the CG's product,
// spmm.cu) and one fused update per term, FP32 vectors with compensated FP32
// dot products combined in FP64 and FP64 series sums, all in a fixed order.
#include <math.h>

#include "gp_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kUpdThreads = 1024;
constexpr unsigned kFull = 0xffffffffu;

struct TaylorState {
  double a;                    // Gershgorin bound of Khat
  double acc[gp::kMaxCols];    // sum_k z_c^T C^k z_c / k so far, per column
};

// Per-block maxima of the absolute row sums of Khat (one warp per row).
__global__ void __launch_bounds__(kThreads) k_gersh(int64_t n, const int64_t* __restrict__ rp,
                                                    const float* __restrict__ val, double* __restrict__ part) {
  __shared__ double sh[kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double best = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * (kThreads / 32) + w; r < n; r += (int64_t)gridDim.x * (kThreads / 32)) {
    double s = 0.0;
    for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += 32) s += fabs((double)val[e]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    best = fmax(best, s);
  }
  if (lane == 0) sh[w] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) m = fmax(m, sh[i]);
    part[blockIdx.x] = m;
  }
}

// a = max of the per-block maxima; the series sums start at zero; the CG
// state is set to "iteration 0, running" so that the SpMM does its work.
__global__ void __launch_bounds__(kThreads) k_taylor_setup(const double* __restrict__ part, int nb, TaylorState* ts,
                                                           gp::CgState* st) {
  __shared__ double sh[kThreads];
  double m = 0.0;
  for (int i = threadIdx.x; i < nb; i += kThreads) m = fmax(m, part[i]);
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ts->a = sh[0];
    st->iter = 0;
    st->fin[0] = 0;
    st->fin[1] = 0;
  }
  if (threadIdx.x < gp::kMaxCols) ts->acc[threadIdx.x] = 0.0;
}

__device__ inline float probe_sign(const uint32_t* __restrict__ zbits, int64_t p, int c, int nv) {
  if (c < 1 || c > nv) return 0.f;
  const uint32_t word = zbits[2 * p + ((c - 1) >> 5)];
  return (word >> ((c - 1) & 31)) & 1u ? -1.f : 1.f;
}

// V_0 = Z: column 1+l holds probe l, the y column and the padding are zero.
__global__ void __launch_bounds__(kThreads) k_taylor_init(int64_t n, int kp, int nv,
                                                          const uint32_t* __restrict__ zbits, float* __restrict__ V) {
  const int64_t total = n * kp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    V[e] = probe_sign(zbits, e / kp, (int)(e % kp), nv);
}

// V <- V - Q / a (so V_k = C V_{k-1} with Q = Khat V_{k-1}), and per-block
// partials of z_c^T V_k.  A thread owns one float4 column slot (the grid
// stride is a multiple of kq) and walks rows; its sums are compensated FP32,
// the block's are combined in FP64 by a fixed tree.
__global__ void __launch_bounds__(kUpdThreads) k_taylor_update(int64_t n, int kq, int nv, const float4* __restrict__ Q,
                                                               float4* __restrict__ V,
                                                               const uint32_t* __restrict__ zbits,
                                                               const TaylorState* ts, double* __restrict__ part) {
  __shared__ double red[kUpdThreads][4];
  const int ny = kUpdThreads / kq;
  const int tx = threadIdx.x % kq, ty = threadIdx.x / kq;
  const float inv_a = (float)(1.0 / ts->a);
  gpd::Dot2 d0, d1, d2, d3;
  if (ty < ny) {
    const int64_t stride = (int64_t)gridDim.x * ny;
    for (int64_t p = (int64_t)blockIdx.x * ny + ty; p < n; p += stride) {
      float4 v = V[p * kq + tx];
      const float4 q = Q[p * kq + tx];
      v.x = fmaf(-inv_a, q.x, v.x);
      v.y = fmaf(-inv_a, q.y, v.y);
      v.z = fmaf(-inv_a, q.z, v.z);
      v.w = fmaf(-inv_a, q.w, v.w);
      V[p * kq + tx] = v;
      d0.add(probe_sign(zbits, p, 4 * tx + 0, nv), v.x);
      d1.add(probe_sign(zbits, p, 4 * tx + 1, nv), v.y);
      d2.add(probe_sign(zbits, p, 4 * tx + 2, nv), v.z);
      d3.add(probe_sign(zbits, p, 4 * tx + 3, nv), v.w);
    }
  }
  red[threadIdx.x][0] = d0.value();
  red[threadIdx.x][1] = d1.value();
  red[threadIdx.x][2] = d2.value();
  red[threadIdx.x][3] = d3.value();
  __syncthreads();
  for (int h = 1; h < ny; h <<= 1) {
    if (ty < ny && (ty & (2 * h - 1)) == 0 && ty + h < ny) {
      const int o = threadIdx.x + h * kq;
#pragma unroll
      for (int q = 0; q < 4; ++q) red[threadIdx.x][q] += red[o][q];
    }
    __syncthreads();
  }
  const int kp = 4 * kq;
  if (threadIdx.x < kp) part[(int64_t)blockIdx.x * kp + threadIdx.x] = red[threadIdx.x / 4][threadIdx.x % 4];
}

// acc_c += (sum over blocks of z_c^T V_k) / k, blocks in a fixed order.
__global__ void __launch_bounds__(kThreads) k_taylor_accum(const double* __restrict__ part, int nb, int kp, int k,
                                                           TaylorState* ts) {
  __shared__ double sh[kThreads];
  const int groups = kThreads / kp;
  const int c = threadIdx.x % kp, g = threadIdx.x / kp;
  double s = 0.0;
  if (g < groups)
    for (int b = g; b < nb; b += groups) s += part[(int64_t)b * kp + c];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < kp) {
    double t = 0.0;
    for (int g2 = 0; g2 < groups; ++g2) t += sh[g2 * kp + threadIdx.x];
    ts->acc[threadIdx.x] += t / (double)k;
  }
}

// Gamma_l = N_act ln a - acc_{1+l}; their mean and sample variance go where
// the SLQ terms go (the likelihood assembly reads them the same way).
__global__ void k_taylor_final(const TaylorState* ts, int nv, int64_t n_act, gp::AsmScalars* s) {
  if (threadIdx.x != 0) return;
  const double a = ts->a;
  const bool ok = a > 0.0 && isfinite(a);
  const double base = ok ? (double)n_act * log(a) : 0.0;
  double mean = 0.0;
  for (int l = 0; l < nv; ++l) mean += base - ts->acc[1 + l];
  mean /= nv;
  double var = 0.0;
  for (int l = 0; l < nv; ++l) {
    const double d = base - ts->acc[1 + l] - mean;
    var += d * d;
  }
  s->slq_mean = mean;
  s->slq_var = nv > 1 ? var / (nv - 1) : 0.0;
  s->status = ok && isfinite(mean) ? GP_OK : GP_ERR_NOT_SPD;
}

}  // namespace

namespace gp {

int taylor_logdet(gp_ctx* c, int nv, int kp, int m) {
  AsmScalars* s = (AsmScalars*)c->asm_s.p;
  const int64_t n = c->n_act;
  if (n == 0) {
    GP_CUDA(cudaMemsetAsync(&s->slq_mean, 0, 2 * sizeof(double), c->stream));
    return GP_OK;
  }
  if (c->precision != GP_FP32_MIXED || kp % 4 || kp > kMaxCols) return GP_ERR_UNSUPPORTED;
  const int kq = kp / 4;
  CgState* st = (CgState*)c->cg.p;
  GP_CHECK(ensure(c, c->taylor, sizeof(TaylorState)));
  TaylorState* ts = (TaylorState*)c->taylor.p;
  const int nb_g = (int)((n + kThreads / 32 - 1) / (kThreads / 32) < (int64_t)c->num_sms * 8
                             ? (n + kThreads / 32 - 1) / (kThreads / 32)
                             : (int64_t)c->num_sms * 8);
  const int ny = kUpdThreads / kq;
  int64_t gu = (n + ny - 1) / ny;
  if (gu > c->num_sms) gu = c->num_sms;
  const int nb_u = (int)gu;
  GP_CHECK(ensure(c, c->part_c, (size_t)(nb_g > nb_u * kp ? nb_g : nb_u * kp) * sizeof(double)));
  double* part = (double*)c->part_c.p;
  k_gersh<<<nb_g, kThreads, 0, c->stream>>>(n, (const int64_t*)c->row_ptr.p, (const float*)c->val.p, part);
  k_taylor_setup<<<1, kThreads, 0, c->stream>>>(part, nb_g, ts, st);
  int64_t gi = (n * kp + kThreads - 1) / kThreads;
  if (gi > (int64_t)c->num_sms * 8) gi = (int64_t)c->num_sms * 8;
  k_taylor_init<<<(unsigned)gi, kThreads, 0, c->stream>>>(n, kp, nv, (const uint32_t*)c->zbits.p, (float*)c->P.p);
  GP_LAUNCH_CHECK();
  c->launches += 3;
  SpmmPlan plan;
  // k = 0: a form that also finishes a CG step leaves every column's state alone
  GP_CHECK(spmm_select(c, kp, c->flags, st, &plan, 0, 0));
  for (int k = 1; k <= m; ++k) {
    spmm_launch(plan, c->stream, c, st);  // Q = Khat V_{k-1}
    k_taylor_update<<<nb_u, kUpdThreads, 0, c->stream>>>(n, kq, nv, (const float4*)c->Q.p, (float4*)c->P.p,
                                                         (const uint32_t*)c->zbits.p, ts, part);
    k_taylor_accum<<<1, kThreads, 0, c->stream>>>(part, nb_u, kp, k, ts);
    GP_LAUNCH_CHECK();
    c->launches += 3;
  }
  k_taylor_final<<<1, 32, 0, c->stream>>>(ts, nv, n, s);
  GP_LAUNCH_CHECK();
  c->launches += 1;
  return GP_OK;
}

}  // namespace gp
