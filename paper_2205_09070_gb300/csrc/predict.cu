// Posterior mean of the GP at test points (Sec. 2.1: the predictive mean at
// x* is kappa^T (K + V)^-1 y with kappa_i = k(x*, x_i) and prior mean 0; here
// V = sigma_n^2 I already sits in K, so alpha = K^-1 y comes from the solver).
//
// k(x*, x_i) = A k~(|x* - x_i| / r_s) sum_m f_m(x*) f_m(x_i) (Eq. eq:bump_kernel
// with Eq. eq:kstat) is non-zero only for training points within r_s of x*
// that share the support of some f_m with it, so each test point scans the
// 3^dim cells around its own cell in the assembled cell list (edge >= r_s,
// Morton-sorted active points).  A test point is not an observation: no noise
// term.  Everything here is FP64: the support tests use the same operation
// order as the assembly's FP64 test; values take 1 - rho^2 and each bump's
// 1 - |x - c|^2 / r^2 without cancellation and sum f_m and sum_m f_m f_m
// compensated; the training side uses the FP64 bump table of the assembly.
#include "gp_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

// One warp per test point q:
//   lane m < n1 sums the bumps of f_m at x*_q in order (support |x-c| < r);
//   the lanes then split the candidates of each neighbour cell, accumulate
//   kappa_qj alpha_j in a fixed order, and the warp adds its lanes' sums by a
//   fixed shuffle tree (deterministic).
__global__ void __launch_bounds__(kThreads) k_predict(const double* __restrict__ xstar, int64_t ns,
                                                      const gp::BumpParam* __restrict__ bumps, int n1, int n2,
                                                      double beta, gp::Grid g, const int2* __restrict__ cells,
                                                      const double* __restrict__ xs,
                                                      const uint32_t* __restrict__ smask,
                                                      const uint32_t* __restrict__ perm,
                                                      const double* __restrict__ F0,
                                                      const double* __restrict__ alpha, double AC, double rs2,
                                                      double rs2l, double inv2l2, double* __restrict__ mean) {
  __shared__ double sF[kWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int dim = g.dim;
  for (int64_t q = (int64_t)blockIdx.x * kWarps + w; q < ns; q += (int64_t)gridDim.x * kWarps) {
    double xq[gp::kMaxDim] = {0.0, 0.0, 0.0};
    for (int k = 0; k < dim; ++k) xq[k] = xstar[q * dim + k];
    double f = 0.0, fc = 0.0;
    bool in_m = false;
    if (lane < n1) {
      for (int j = 0; j < n2; ++j) {
        const gp::BumpParam& bp = bumps[lane * n2 + j];
        double d2 = 0.0;
        for (int k = 0; k < dim; ++k) {
          const double t = __dsub_rn(xq[k], bp.c[k]);
          d2 = __dadd_rn(d2, __dmul_rn(t, t));
        }
        const double qq = __ddiv_rn(d2, bp.r2);
        if (qq < 1.0) {
          // value from u = 1 - q without cancellation, summed compensated
          const double u = gpd::one_minus_ratio(xq, bp.c, dim, bp.r2, bp.r2l);
          if (u > 0.0) {
            double t, e;
            gpd::two_sum(f, bp.a * exp(beta - beta / u), t, e);
            f = t;
            fc += e;
          }
          in_m = true;
        }
      }
    }
    f += fc;
    const uint32_t mq = __ballot_sync(kFull, in_m);  // bit m: x*_q inside some bump of f_m
    sF[w][lane] = f;
    __syncwarp();
    double acc = 0.0;
    if (mq != 0u) {
      int c[gp::kMaxDim];
      gpd::cell_of(xq, g, c);
      int nst = 1;
      for (int k = 0; k < dim; ++k) nst *= 3;
      for (int s = 0; s < nst; ++s) {
        int t = s;
        bool ok = true;
        int64_t lin = 0, mult = 1;
        for (int k = 0; k < dim; ++k) {
          const int cc = c[k] + t % 3 - 1;
          t /= 3;
          ok = ok && cc >= 0 && cc < g.G[k];
          lin += (int64_t)cc * mult;
          mult *= g.G[k];
        }
        if (!ok) continue;
        const int2 se = cells[lin];
        for (int j = se.x + lane; j < se.y; j += 32) {
          uint32_t common = mq & smask[j];
          if (common == 0u) continue;
          double d2 = 0.0;
          for (int k = 0; k < dim; ++k) {
            const double t2 = __dsub_rn(xq[k], xs[(int64_t)j * dim + k]);
            d2 = __dadd_rn(d2, __dmul_rn(t2, t2));
          }
          if (!(d2 < rs2)) continue;
          const uint32_t i = perm[j];
          const double S = gpd::dot2_bits(sF[w], F0 + (int64_t)i * n1, common);
          double s2 = (rs2 - d2) / rs2;
          if (s2 < 1e-2) s2 = gpd::one_minus_ratio(xq, xs + (int64_t)j * dim, dim, rs2, rs2l);
          double kst = s2 > 0.0 ? gpd::kstat_unit_d(d2 / rs2, s2) : 0.0;
          if (inv2l2 > 0.0) kst *= exp(-d2 * inv2l2);
          acc += AC * kst * S * alpha[i];
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lane == 0) mean[q] = acc;
    __syncwarp();  // sF[w] is rewritten by the next test point
  }
}

// Posterior variance (Sec. 2.1, Eq. eq:pred_distr: the covariance at x* is
// k(x*, x*) - kappa^T (K + V)^-1 kappa).  One warp per test point q of a block
// of nq points (the block's column q): the prior variance k(x*_q, x*_q) =
// A C sum_m f_m(x*_q)^2 (k~(0) = C, k_c(x, x) = 1) into prior[q] and, unless B
// is null, the right-hand side column B[j, q] = D_j^-1/2 k(x*_q, x_j) /
// sqrt(k(x*_q, x*_q)) for the active training points j (Morton order) in
// support, entries at j ldr + q ldc.  The scale makes every entry at most 1
// (Cauchy-Schwarz: |k(x*, x_j)| <= sqrt(k(x*, x*) K_jj), K_jj <= D_j), so
// columns of test points far out on a bump's flank, whose kappa is tiny, do
// not underflow in FP32; CG is indifferent to a column's scale, and
// var = k(x*, x*) (1 - b^T Khat^-1 b) for the scaled column b.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pred_rhs(const double* __restrict__ xstar, int nq,
                                                       const gp::BumpParam* __restrict__ bumps, int n1, int n2,
                                                       double beta, gp::Grid g, const int2* __restrict__ cells,
                                                       const double* __restrict__ xs,
                                                       const uint32_t* __restrict__ smask,
                                                       const uint32_t* __restrict__ perm,
                                                       const double* __restrict__ F0,
                                                       const double* __restrict__ dinv64, double AC, double rs2,
                                                       double rs2l, double inv2l2, int dim, T* __restrict__ B,
                                                       int64_t ldr, int64_t ldc, double* __restrict__ prior) {
  __shared__ double sF[kWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = blockIdx.x * kWarps + w; q < nq; q += gridDim.x * kWarps) {
    double xq[gp::kMaxDim] = {0.0, 0.0, 0.0};
    for (int k = 0; k < dim; ++k) xq[k] = xstar[(int64_t)q * dim + k];
    double f = 0.0, fc = 0.0;
    bool in_m = false;
    if (lane < n1) {
      for (int j = 0; j < n2; ++j) {
        const gp::BumpParam& bp = bumps[lane * n2 + j];
        double d2 = 0.0;
        for (int k = 0; k < dim; ++k) {
          const double t = __dsub_rn(xq[k], bp.c[k]);
          d2 = __dadd_rn(d2, __dmul_rn(t, t));
        }
        if (__ddiv_rn(d2, bp.r2) < 1.0) {
          const double u = gpd::one_minus_ratio(xq, bp.c, dim, bp.r2, bp.r2l);
          if (u > 0.0) {
            double t, e;
            gpd::two_sum(f, bp.a * exp(beta - beta / u), t, e);
            f = t;
            fc += e;
          }
          in_m = true;
        }
      }
    }
    f += fc;
    const uint32_t mq = __ballot_sync(kFull, in_m);
    sF[w][lane] = f;
    __syncwarp();
    const double pr = AC * gpd::dot2_bits(sF[w], sF[w], mq);
    if (lane == 0) prior[q] = pr;
    const double inv_s = pr > 0.0 ? 1.0 / sqrt(pr) : 0.0;
    if (B && mq != 0u && pr > 0.0) {
      int c[gp::kMaxDim];
      gpd::cell_of(xq, g, c);
      int nst = 1;
      for (int k = 0; k < dim; ++k) nst *= 3;
      for (int s = 0; s < nst; ++s) {
        int t = s;
        bool ok = true;
        int64_t lin = 0, mult = 1;
        for (int k = 0; k < dim; ++k) {
          const int cc = c[k] + t % 3 - 1;
          t /= 3;
          ok = ok && cc >= 0 && cc < g.G[k];
          lin += (int64_t)cc * mult;
          mult *= g.G[k];
        }
        if (!ok) continue;
        const int2 se = cells[lin];
        for (int j = se.x + lane; j < se.y; j += 32) {
          const uint32_t common = mq & smask[j];
          if (common == 0u) continue;
          double d2 = 0.0;
          for (int k = 0; k < dim; ++k) {
            const double t2 = __dsub_rn(xq[k], xs[(int64_t)j * dim + k]);
            d2 = __dadd_rn(d2, __dmul_rn(t2, t2));
          }
          if (!(d2 < rs2)) continue;
          const double S = gpd::dot2_bits(sF[w], F0 + (int64_t)perm[j] * n1, common);
          double s2 = (rs2 - d2) / rs2;
          if (s2 < 1e-2) s2 = gpd::one_minus_ratio(xq, xs + (int64_t)j * dim, dim, rs2, rs2l);
          double kst = s2 > 0.0 ? gpd::kstat_unit_d(d2 / rs2, s2) : 0.0;
          if (inv2l2 > 0.0) kst *= exp(-d2 * inv2l2);
          B[(int64_t)j * ldr + (int64_t)q * ldc] = (T)(AC * kst * S * dinv64[j] * inv_s);
        }
      }
    }
    __syncwarp();  // sF[w] is rewritten by the next test point
  }
}

// var[q] = prior[q] (1 - sum_j B[j, q] X[j, q]) for the FP32 block (row-major,
// kq float4 slots per row): thread per slot, rows strided, compensated sums,
// per-block partials in a fixed order; the last block finishes the columns.
constexpr int kVarThreads = 1024;
__global__ void __launch_bounds__(kVarThreads) k_var_f32(int64_t n, int kq, int nq, const float4* __restrict__ B,
                                                         const float4* __restrict__ X, const double* __restrict__ prior,
                                                         double* __restrict__ var, double* __restrict__ part,
                                                         unsigned* ticket) {
  __shared__ double red[kVarThreads][4];
  __shared__ bool last;
  const int ny = kVarThreads / kq;
  const int tx = threadIdx.x % kq, ty = threadIdx.x / kq;
  gpd::Dot2 d0, d1, d2, d3;
  if (ty < ny) {
    for (int64_t p = (int64_t)blockIdx.x * ny + ty; p < n; p += (int64_t)gridDim.x * ny) {
      const float4 b = B[p * kq + tx], x = X[p * kq + tx];
      d0.add(b.x, x.x);
      d1.add(b.y, x.y);
      d2.add(b.z, x.z);
      d3.add(b.w, x.w);
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
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicInc(ticket, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < nq) {
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(part + (int64_t)b * kp + threadIdx.x);
    var[threadIdx.x] = prior[threadIdx.x] * (1.0 - t);
  }
}

// The same for the FP64 block (column-major, column q contiguous): one block
// per column, compensated sums, a fixed-order tree.
__global__ void __launch_bounds__(kThreads) k_var_f64(int64_t n, const double* __restrict__ B,
                                                      const double* __restrict__ X, const double* __restrict__ prior,
                                                      double* __restrict__ var) {
  __shared__ double sh[kThreads];
  const int q = blockIdx.x;
  double s = 0.0, c = 0.0;
  for (int64_t p = threadIdx.x; p < n; p += kThreads) {
    double pr, pe, t, te;
    gpd::two_prod(B[(int64_t)q * n + p], X[(int64_t)q * n + p], pr, pe);
    gpd::two_sum(s, pr, t, te);
    s = t;
    c += te + pe;
  }
  sh[threadIdx.x] = s + c;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) var[q] = prior[q] * (1.0 - sh[0]);
}

}  // namespace

namespace gp {

int predict_var(gp_ctx* c, const double* xstar, int64_t ns, double* var, const gp_opts* o, int* iters_out,
                double* max_rel) {
  *iters_out = 0;
  *max_rel = 0.0;
  if (ns == 0) return GP_OK;
  constexpr int kBlock = 64;  // test points per right-hand-side block (<= kMaxCols)
  const double inv2l2 = c->core == GP_CORE_SQEXP ? 1.0 / (2.0 * c->ell * c->ell) : 0.0;
  double rs2, rs2l;
  gpd::two_prod(c->r_s, c->r_s, rs2, rs2l);
  const double AC = c->A * kStatPrefactor;
  const int64_t n = c->n_act;
  GP_CHECK(ensure(c, c->pv_prior, (size_t)kBlock * sizeof(double)));
  if (n == 0) {
    // no active training point: kappa = 0, the variance is the prior's
    for (int64_t q0 = 0; q0 < ns; q0 += kBlock) {
      const int nq = (int)(ns - q0 < kBlock ? ns - q0 : kBlock);
      k_pred_rhs<double><<<(nq + kWarps - 1) / kWarps, kThreads, 0, c->stream>>>(
          xstar + q0 * c->dim, nq, (const gp::BumpParam*)c->bump.p, c->n1, c->n2, c->beta, c->grid, nullptr,
          nullptr, nullptr, nullptr, nullptr, nullptr, AC, rs2, rs2l, inv2l2, c->dim, (double*)nullptr, 0, 0,
          var + q0);
      GP_LAUNCH_CHECK();
      c->launches += 1;
    }
    return GP_OK;
  }
  GP_CHECK(precond_setup(c, o->precond_block));
  int status = GP_OK;
  for (int64_t q0 = 0; q0 < ns; q0 += kBlock) {
    const int nq = (int)(ns - q0 < kBlock ? ns - q0 : kBlock);
    const unsigned gq = (unsigned)((nq + kWarps - 1) / kWarps);
    int iters = 0;
    double mr = 0.0;
    int st;
    if (c->precision == GP_FP64) {
      GP_CHECK(ensure(c, c->pv_B, (size_t)n * nq * sizeof(double)));
      GP_CUDA(cudaMemsetAsync(c->pv_B.p, 0, (size_t)n * nq * sizeof(double), c->stream));
      k_pred_rhs<double><<<gq, kThreads, 0, c->stream>>>(
          xstar + q0 * c->dim, nq, (const gp::BumpParam*)c->bump.p, c->n1, c->n2, c->beta, c->grid,
          (const int2*)c->cells.p, (const double*)c->xs.p, (const uint32_t*)c->smask.p, (const uint32_t*)c->vals.p,
          (const double*)c->F0.p, (const double*)c->dinv64.p, AC, rs2, rs2l, inv2l2, c->dim, (double*)c->pv_B.p, 1,
          n, (double*)c->pv_prior.p);
      GP_LAUNCH_CHECK();
      c->launches += 1;
      st = cg_run_fp64(c, nq, nullptr, 0, o->seed, 0, o->max_iter, o->cg_rtol, o->check_every, &iters, &mr,
                       (const double*)c->pv_B.p);
      if (st != GP_OK && st != GP_ERR_NOT_CONVERGED) return st;
      k_var_f64<<<nq, kThreads, 0, c->stream>>>(n, (const double*)c->pv_B.p, (const double*)c->X.p,
                                                (const double*)c->pv_prior.p, var + q0);
    } else {
      const int kp = (nq + 3) / 4 * 4;
      GP_CHECK(ensure(c, c->pv_B, (size_t)n * kp * sizeof(float)));
      GP_CUDA(cudaMemsetAsync(c->pv_B.p, 0, (size_t)n * kp * sizeof(float), c->stream));
      k_pred_rhs<float><<<gq, kThreads, 0, c->stream>>>(
          xstar + q0 * c->dim, nq, (const gp::BumpParam*)c->bump.p, c->n1, c->n2, c->beta, c->grid,
          (const int2*)c->cells.p, (const double*)c->xs.p, (const uint32_t*)c->smask.p, (const uint32_t*)c->vals.p,
          (const double*)c->F0.p, (const double*)c->dinv64.p, AC, rs2, rs2l, inv2l2, c->dim, (float*)c->pv_B.p, kp,
          1, (double*)c->pv_prior.p);
      GP_LAUNCH_CHECK();
      c->launches += 1;
      st = cg_run(c, nq, kp, nullptr, 0, o->seed, 0, o->max_iter, o->cg_rtol, o->check_every, &iters, &mr,
                  c->pc_block > 0, false, (const float*)c->pv_B.p);
      if (st != GP_OK && st != GP_ERR_NOT_CONVERGED) return st;
      const int kq = kp / 4;
      int64_t gv = (n + kVarThreads / kq - 1) / (kVarThreads / kq);
      if (gv > c->num_sms) gv = c->num_sms;
      if (gv < 1) gv = 1;
      GP_CHECK(ensure(c, c->part_c, (size_t)gv * kp * sizeof(double)));
      k_var_f32<<<(unsigned)gv, kVarThreads, 0, c->stream>>>(n, kq, nq, (const float4*)c->pv_B.p,
                                                             (const float4*)c->X.p, (const double*)c->pv_prior.p,
                                                             var + q0, (double*)c->part_c.p,
                                                             &((gp::AsmScalars*)c->asm_s.p)->ticket5);
    }
    GP_LAUNCH_CHECK();
    c->launches += 1;
    if (st == GP_ERR_NOT_CONVERGED) status = st;
    *iters_out = iters > *iters_out ? iters : *iters_out;
    *max_rel = mr > *max_rel ? mr : *max_rel;
  }
  return status;
}

int predict_mean(gp_ctx* c, const double* xstar, int64_t ns, const double* alpha, double* mean) {
  if (ns == 0) return GP_OK;
  if (c->n_act == 0) {
    // no training point lies in any bump: kappa = 0 for every test point
    GP_CUDA(cudaMemsetAsync(mean, 0, (size_t)ns * sizeof(double), c->stream));
    return GP_OK;
  }
  double rs2, rs2l;
  gpd::two_prod(c->r_s, c->r_s, rs2, rs2l);
  int64_t blocks = (ns + kWarps - 1) / kWarps;
  if (blocks > (int64_t)c->num_sms * 16) blocks = (int64_t)c->num_sms * 16;
  k_predict<<<(unsigned)blocks, kThreads, 0, c->stream>>>(
      xstar, ns, (const gp::BumpParam*)c->bump.p, c->n1, c->n2, c->beta, c->grid, (const int2*)c->cells.p,
      (const double*)c->xs.p, (const uint32_t*)c->smask.p, (const uint32_t*)c->vals.p, (const double*)c->F0.p,
      alpha, c->A * kStatPrefactor, rs2, rs2l,
      c->core == GP_CORE_SQEXP ? 1.0 / (2.0 * c->ell * c->ell) : 0.0, mean);
  GP_LAUNCH_CHECK();
  c->launches += 1;
  return GP_OK;
}

}  // namespace gp
