// Analytic gradient of ln L (Sec. 2.1, Eq. eqn:log_likelihood) with respect to
// every hyperparameter, without ever storing dK/dh:
//   d ln L / d theta = sum_ij W_ij dK_ij/d theta,
//   W_ij = 1/2 alpha_i alpha_j - 1/(4 nv) sum_l (u_li z_lj + z_li u_lj),
// alpha = K^-1 y, u_l = K^-1 D^1/2 zhat_l, z_l = D^-1/2 zhat_l (Hutchinson's
// estimator of tr(K^-1 dK) on the Jacobi-scaled probes).  With
// K_ij = A k~(d_ij; r_s) S_ij + sigma_n^2 [i=j], S_ij = sum_m F_im F_jm
// (Eq. eq:bump_kernel):
//   dK/dA      = k~ S
//   dK/dr_s    = A (6C/r_s) rho^2 (atanh s - s) S      (differentiating Eq. eq:kstat)
//   dK/dsigma2 = I
//   dK/dtheta_mb = A k~ (dphi_mb(x_i) F_jm + F_im dphi_mb(x_j)), so
//   d ln L / d theta_mb = 2 sum_i dphi_mb(x_i)/d theta g_im,  g_im = sum_j W_ij A k~_ij F_jm.
// k_adjoint walks the CSR pattern (one warp per row, one lane per stored
// entry) and recomputes k~ and its r_s-derivative from the coordinates;
// k_bump_grad contracts g with the bump derivatives of Eq. eq:bump.
#include <math.h>

#include "gp_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr double kPrefactor = 0.26596152026762182;  // sqrt(2) / (3 sqrt(pi))

struct AdjArgs {
  int64_t n;
  int dim, n1, nv;
  int64_t ld;            // row stride (row-major) or column stride (column-major) of X
  const int64_t* rp;
  const int32_t* col;
  const int4* cellc;
  const float4* xr;
  const double* xs;
  const float2* xhl;     // FP32 path: coordinates as double-float pairs
  const void* Fs;
  const uint32_t* mask;
  const void* dinv;
  const void* X;
  const uint32_t* zbits;
  void* g;               // n x n1
  double* part;          // grid x 3
  gp::AsmScalars* s;
  float scale;           // (h / r_s)^2
  double rs2, AC, dk_coef;  // r_s^2, A C, A (6 C / r_s)
  double C;
  double inv2l2;            // 1 / (2 l^2) of the squared-exponential core, 0 without one
  double inv_l;             // 1 / l
  float rs2h, rs2lo, inv_rs2f;  // FP32 path: r_s^2 as a pair, 1 / r_s^2
};

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <typename T, bool COLMAJOR>
__device__ inline T xval(const T* X, int64_t ld, int64_t row, int c) {
  return COLMAJOR ? X[(int64_t)c * ld + row] : X[row * ld + c];
}

template <typename T, bool COLMAJOR>
__global__ void __launch_bounds__(kThreads) k_adjoint(AdjArgs a) {
  extern __shared__ unsigned char smem_raw[];
  // per warp: u_i (nv values) then per-lane slots for g (32 x n1)
  T* sh = (T*)smem_raw;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T* sh_u = sh + (size_t)w * (gp::kMaxProbes + 32 * a.n1);
  T* slot = sh_u + gp::kMaxProbes;
  const T* X = (const T*)a.X;
  const T* Fs = (const T*)a.Fs;
  const T* dinv = (const T*)a.dinv;
  T* g = (T*)a.g;
  double accA = 0.0, accR = 0.0, accS = 0.0, accL = 0.0;
  for (int q = lane; q < 32 * a.n1; q += 32) slot[q] = 0;
  for (int64_t p = (int64_t)blockIdx.x * kWarps + w; p < a.n; p += (int64_t)gridDim.x * kWarps) {
    const uint32_t mi = a.mask[p];
    const T di = dinv[p];
    const T al_i = di * xval<T, COLMAJOR>(X, a.ld, p, 0);
    for (int l = lane; l < a.nv; l += 32) sh_u[l] = xval<T, COLMAJOR>(X, a.ld, p, 1 + l);
    const uint32_t zi0 = a.zbits[2 * p], zi1 = a.zbits[2 * p + 1];
    const int4 ci = a.cellc[p];
    const float4 xi = a.xr[p];
    __syncwarp();
    T rA = 0, rR = 0, rS = 0, rL = 0;
    for (int64_t e = a.rp[p] + lane; e < a.rp[p + 1]; e += 32) {
      const int j = a.col[e];
      const uint32_t mj = a.mask[j];
      T rho2, s2;
      if (sizeof(T) == 4) {
        const int4 cj = a.cellc[j];
        const float4 xj = a.xr[j];
        const float dx = (xj.x + (float)(cj.x - ci.x)) - xi.x;
        const float dy = (xj.y + (float)(cj.y - ci.y)) - xi.y;
        const float dz = (xj.z + (float)(cj.z - ci.z)) - xi.z;
        const float r2 = (dx * dx + dy * dy + dz * dz) * a.scale;
        rho2 = (T)r2;
        s2 = (T)(1.0f - r2);
        if (s2 < (T)0.1) {
          // near the edge: d^2 and r_s^2 - d^2 from the double-float
          // coordinates (as in the pair fill), in FP32 arithmetic
          float eh, el;
          gpd::dist2_pair_f(a.xhl, a.dim, p, j, eh, el);
          rho2 = (T)((eh + el) * a.inv_rs2f);
          s2 = (T)(gpd::pair_gap_f(a.rs2h, a.rs2lo, eh, el) * a.inv_rs2f);
        }
      } else {
        double e2 = 0.0;
        for (int k = 0; k < a.dim; ++k) {
          const double t = a.xs[p * a.dim + k] - a.xs[(int64_t)j * a.dim + k];
          e2 += t * t;
        }
        rho2 = (T)(e2 / a.rs2);
        s2 = (T)((a.rs2 - e2) / a.rs2);
      }
      if (s2 <= (T)0) s2 = (T)0;
      T kt = s2 > (T)0 ? gpd::Real<T>::kstat(rho2, s2) : (T)0;
      T dk = s2 > (T)0 ? gpd::Real<T>::dk(rho2, s2) : (T)0;
      // squared-exponential core: every term of dK carries k_c, and
      // dK/dl = K_s d^2 / l^3 (d^2 = rho^2 r_s^2)
      T kc = (T)1, d2l3 = (T)0;
      if (a.inv2l2 > 0.0) {
        const double d2 = (double)rho2 * a.rs2;
        kc = (T)gpd::sqexp_core<T>(d2 * a.inv2l2);
        d2l3 = (T)(d2 * a.inv_l * a.inv_l * a.inv_l);
        kt *= kc;
        dk *= kc;
      }
      const T dj = dinv[j];
      const T al_j = dj * xval<T, COLMAJOR>(X, a.ld, j, 0);
      const uint32_t zj0 = a.zbits[2 * (int64_t)j], zj1 = a.zbits[2 * (int64_t)j + 1];
      T t1 = 0, t2 = 0;
      for (int l = 0; l < a.nv; ++l) {
        const uint32_t bj = (l < 32 ? zj0 >> l : zj1 >> (l - 32)) & 1u;
        const uint32_t bi = (l < 32 ? zi0 >> l : zi1 >> (l - 32)) & 1u;
        const T ui = sh_u[l];
        const T uj = xval<T, COLMAJOR>(X, a.ld, j, 1 + l);
        t1 += bj ? -ui : ui;
        t2 += bi ? -uj : uj;
      }
      const T W = (T)0.5 * al_i * al_j - (T)(0.25 / a.nv) * di * dj * (t1 + t2);
      T S = 0;
      uint32_t common = mi & mj;
      while (common) {
        const int m = __ffs(common) - 1;
        common &= common - 1u;
        const T fj = Fs[(int64_t)j * a.n1 + m];
        S += Fs[p * a.n1 + m] * fj;
        slot[lane * a.n1 + m] += W * (T)a.AC * kt * fj;
      }
      rA += W * (T)a.C * kt * S;
      rR += W * (T)a.dk_coef * rho2 * dk * S;
      rL += W * (T)a.AC * kt * S * d2l3;
      if (j == p) rS += W;
    }
    accA += warp_sum_d((double)rA);
    accR += warp_sum_d((double)rR);
    accS += warp_sum_d((double)rS);
    accL += warp_sum_d((double)rL);
    __syncwarp();
    for (int m = lane; m < a.n1; m += 32) {
      T t = 0;
      for (int l = 0; l < 32; ++l) {
        t += slot[l * a.n1 + m];
        slot[l * a.n1 + m] = 0;
      }
      g[p * a.n1 + m] = t;
    }
    __syncwarp();
  }
  __shared__ double red[kWarps][4];
  __shared__ bool last;
  if (lane == 0) {
    red[w][0] = accA;
    red[w][1] = accR;
    red[w][2] = accS;
    red[w][3] = accL;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int ww = 0; ww < kWarps; ++ww) t += red[ww][threadIdx.x];
    a.part[blockIdx.x * 4 + threadIdx.x] = t;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicInc(&a.s->ticket0, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x < 4) {
    __threadfence();
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(a.part + b * 4 + threadIdx.x);
    if (threadIdx.x == 0) a.s->grad_A = t;
    if (threadIdx.x == 1) a.s->grad_rs = t;
    if (threadIdx.x == 2) a.s->grad_s2 = t;
    if (threadIdx.x == 3) a.s->grad_l = t;
  }
}

// d ln L / d theta_mb = 2 sum_i g_im d phi_mb(x_i) / d theta  for
// theta in (centre_k, r, a); one lane per active row, bumps visited in order,
// warp sums into warp-private shared slots, then fixed-order block and grid sums.
// phi = a exp(beta - beta/u), q = |x - c|^2 / r^2, u = 1 - q:
//   dphi/dc_k = 2 beta phi (x_k - c_k) / (r^2 u^2), dphi/dr = 2 beta phi q / (r u^2),
//   dphi/da = exp(beta - beta/u).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bump_grad(int64_t n, int dim, int n1, int n2, double beta,
                                                        const gp::BumpParam* __restrict__ bumps,
                                                        const double* __restrict__ xs, const double* __restrict__ lo,
                                                        const uint32_t* __restrict__ mask, const T* __restrict__ g,
                                                        double* __restrict__ part, double* __restrict__ out,
                                                        gp::AsmScalars* s) {
  extern __shared__ double acc[];  // kWarps x nb x (dim+2)
  const int nb = n1 * n2, np = dim + 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < kWarps * nb * np; q += blockDim.x) acc[q] = 0.0;
  __syncthreads();
  double* wacc = acc + (size_t)w * nb * np;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t base = (int64_t)blockIdx.x * kThreads + w * 32; base < n; base += stride) {
    const int64_t p = base + lane;
    const bool valid = p < n;
    const uint32_t mi = valid ? mask[p] : 0u;
    double xi[gp::kMaxDim] = {0, 0, 0};
    float x32[gp::kMaxDim] = {0, 0, 0};
    if (valid)
      for (int k = 0; k < dim; ++k) {
        xi[k] = xs[p * dim + k];
        x32[k] = (float)(xi[k] - lo[k]);
      }
    for (int b = 0; b < nb; ++b) {
      const gp::BumpParam& bp = bumps[b];
      const bool cand_m = (mi >> bp.m) & 1u;
      if (__ballot_sync(kFull, cand_m) == 0u) continue;
      double v[gp::kMaxDim + 2] = {0, 0, 0, 0, 0};
      if (cand_m) {
        float q32 = 0.0f;
        for (int k = 0; k < dim; ++k) {
          const float t = x32[k] - bp.c32[k];
          q32 = fmaf(t, t, q32);
        }
        q32 *= bp.inv_r2_32;
        if (q32 < 1.0f + bp.margin) {
          double d2 = 0.0;
          for (int k = 0; k < dim; ++k) {
            const double t = __dsub_rn(xi[k], bp.c[k]);
            d2 = __dadd_rn(d2, __dmul_rn(t, t));
          }
          const double q = __ddiv_rn(d2, bp.r2);
          if (q < 1.0) {
            const double u = 1.0 - q;
            const double ex = exp(beta - beta / u);
            const double phi = bp.a * ex;
            const double gi = 2.0 * (double)g[p * n1 + bp.m];
            const double cc = 2.0 * beta * phi / (bp.r2 * u * u);
            for (int k = 0; k < dim; ++k) v[k] = gi * cc * (xi[k] - bp.c[k]);
            v[dim] = gi * 2.0 * beta * phi * q / (bp.r * u * u);
            v[dim + 1] = gi * ex;
          }
        }
      }
      for (int t = 0; t < np; ++t) {
        const double r = warp_sum_d(v[t]);
        if (lane == 0) wacc[b * np + t] += r;
      }
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nb * np; q += blockDim.x) {
    double t = 0.0;
    for (int ww = 0; ww < kWarps; ++ww) t += acc[(size_t)ww * nb * np + q];
    part[(int64_t)blockIdx.x * nb * np + q] = t;
  }
  __threadfence();
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicInc(&s->ticket1, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    for (int q = threadIdx.x; q < nb * np; q += blockDim.x) {
      double t = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(part + (int64_t)b * nb * np + q);
      out[q] = t;
    }
  }
}

unsigned grid_for(int64_t items, int per_block, int max_blocks) {
  int64_t gg = (items + per_block - 1) / per_block;
  if (gg < 1) gg = 1;
  if (gg > max_blocks) gg = max_blocks;
  return (unsigned)gg;
}

template <typename T, bool COLMAJOR>
int run_adjoint(gp_ctx* c, int nv, int64_t ld) {
  const int64_t n = c->n_act;
  gp::AsmScalars* s = (gp::AsmScalars*)c->asm_s.p;
  const int nb = c->nb, np = c->dim + 2;
  GP_CHECK(gp::ensure(c, c->g, (size_t)n * c->n1 * sizeof(T)));
  const unsigned gw = grid_for(n, kWarps, c->num_sms * 4);
  GP_CHECK(gp::ensure(c, c->part_c, (size_t)gw * 4 * sizeof(double)));
  AdjArgs a{};
  a.n = n;
  a.dim = c->dim;
  a.n1 = c->n1;
  a.nv = nv;
  a.ld = ld;
  a.rp = (const int64_t*)c->row_ptr.p;
  a.col = (const int32_t*)c->col.p;
  a.cellc = (const int4*)c->cellc.p;
  a.xr = (const float4*)c->xr.p;
  a.xs = (const double*)c->xs.p;
  a.Fs = c->Fs.p;
  a.mask = (const uint32_t*)c->smask.p;
  a.dinv = c->dinv.p;
  a.X = c->X.p;
  a.zbits = (const uint32_t*)c->zbits.p;
  a.g = c->g.p;
  a.part = (double*)c->part_c.p;
  a.s = s;
  const double sc = (c->grid.h / c->r_s) * (c->grid.h / c->r_s);
  a.scale = (float)sc;
  a.rs2 = c->r_s * c->r_s;
  a.xhl = (const float2*)c->xhl.p;
  a.rs2h = (float)a.rs2;
  a.rs2lo = (float)((a.rs2 - (double)a.rs2h) + fma(c->r_s, c->r_s, -a.rs2));
  a.inv_rs2f = (float)(1.0 / a.rs2);
  a.C = kPrefactor;
  a.AC = c->A * kPrefactor;
  a.dk_coef = c->A * 6.0 * kPrefactor / c->r_s;
  a.inv2l2 = c->core == GP_CORE_SQEXP ? 1.0 / (2.0 * c->ell * c->ell) : 0.0;
  a.inv_l = c->core == GP_CORE_SQEXP ? 1.0 / c->ell : 0.0;
  const size_t smem = (size_t)kWarps * (gp::kMaxProbes + 32 * c->n1) * sizeof(T);
  GP_CUDA(cudaFuncSetAttribute(k_adjoint<T, COLMAJOR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const bool timed = (c->flags & GP_FLAG_TIME_KERNELS) != 0;
  if (timed) {
    GP_CHECK(gp::kernel_events(c));
    GP_CUDA(cudaEventRecord(c->kev[130], c->stream));
  }
  k_adjoint<T, COLMAJOR><<<gw, kThreads, smem, c->stream>>>(a);
  GP_LAUNCH_CHECK();
  if (timed) GP_CUDA(cudaEventRecord(c->kev[131], c->stream));
  c->launches += 1;

  // bump derivatives
  GP_CHECK(gp::ensure(c, c->grad_bump, (size_t)nb * np * sizeof(double)));
  GP_CHECK(gp::ensure(c, c->out_tmp, 4 * sizeof(double)));
  GP_CHECK(gp::ensure_pinned(c, 4 * sizeof(double)));
  double* lo_h = (double*)c->pinned;
  for (int k = 0; k < 3; ++k) lo_h[k] = k < c->dim ? c->grid.lo[k] : 0.0;
  GP_CUDA(cudaMemcpyAsync(c->out_tmp.p, lo_h, 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  const unsigned gb = grid_for(n, kThreads, c->num_sms * 2);
  GP_CHECK(gp::ensure(c, c->grad_part, (size_t)gb * nb * np * sizeof(double)));
  const size_t smem2 = (size_t)kWarps * nb * np * sizeof(double);
  GP_CUDA(cudaFuncSetAttribute(k_bump_grad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
  k_bump_grad<T><<<gb, kThreads, smem2, c->stream>>>(n, c->dim, c->n1, c->n2, c->beta,
                                                     (const gp::BumpParam*)c->bump.p, (const double*)c->xs.p,
                                                     (const double*)c->out_tmp.p, (const uint32_t*)c->smask.p,
                                                     (const T*)c->g.p, (double*)c->grad_part.p,
                                                     (double*)c->grad_bump.p, s);
  GP_LAUNCH_CHECK();
  c->launches += 1;
  // the pinned lo values must stay intact until the copy above has run
  GP_CUDA(cudaStreamSynchronize(c->stream));
  if (timed) c->t_adj += gp::event_ms(c->kev[130], c->kev[131]);
  return GP_OK;
}

}  // namespace

namespace gp {

int adjoint(gp_ctx* c, int nv, int kp) {
  if (c->n_act == 0) return GP_OK;
  if (c->precision == GP_FP64) return run_adjoint<double, true>(c, nv, c->n_act);
  return run_adjoint<float, false>(c, nv, kp);
}

}  // namespace gp
