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

}  // namespace

namespace gp {

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
