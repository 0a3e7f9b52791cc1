// Block-Jacobi preconditioner of the FP32 batched CG.
//
// The active rows are in Morton / sub-cell order, so B consecutive rows are
// close in space and strongly coupled.  M = blockdiag(Khat_bb) over blocks of
// B consecutive rows (B = 8, 16, 32, 64 or 128); each block is factored
// (FP64 for B <= 32, FP32 for 64 and 128; one CTA of B threads per block,
// Cholesky M_bb = L L^T, then M_bb^-1 = L^-T L^-1) and M^-1 is stored in FP32,
// B x B row-major per block, zero outside the block's rows for the last,
// shorter block.  Preconditioning changes only how fast CG converges: the
// solves Khat u = b it feeds are the same.
#include <math.h>

#include "gp_internal.cuh"

namespace {

// One CTA of B threads per diagonal block (grid-stride); thread i owns row i
// of the block.  A (the block of Khat, overwritten by L; FP64) and Y = L^-1
// live in dynamic shared memory, B x (B+1) entries each (B <= 32; larger
// blocks take the FP32 set-up below).
template <int B>
__global__ void __launch_bounds__(B) k_pc_setup(int64_t n, int64_t nblk, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ col, const float* __restrict__ val,
                                                float* __restrict__ Mout, int* __restrict__ part,
                                                gp::AsmScalars* s) {
  extern __shared__ double pc_sm[];
  double (*A)[B + 1] = (double (*)[B + 1])pc_sm;
  double (*Y)[B + 1] = (double (*)[B + 1])(pc_sm + B * (B + 1));
  __shared__ int bad_any;
  const int t = threadIdx.x;
  if (t == 0) bad_any = 0;
  int bad = 0;
  for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int64_t r0 = b * B;
    const int nb = (int)min((int64_t)B, n - r0);
    for (int j = 0; j < B; ++j) A[t][j] = 0.0;
    if (t < nb) {
      const int64_t row = r0 + t;
      for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
        const int64_t j = col[e];
        if (j >= r0 && j < r0 + nb) A[t][j - r0] = (double)val[e];
      }
    }
    __syncthreads();
    // Cholesky, column by column (dot-product form, lower triangle only)
    for (int j = 0; j < nb; ++j) {
      if (t == j) {
        double d = A[j][j];
        for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
        if (!(d > 0.0)) {
          bad = 1;
          d = 1.0;
        }
        A[j][j] = sqrt(d);
      }
      __syncthreads();
      if (t > j && t < nb) {
        double v = A[t][j];
        for (int k = 0; k < j; ++k) v -= A[t][k] * A[j][k];
        A[t][j] = v / A[j][j];
      }
      __syncthreads();
    }
    // Y = L^-1, thread c computes column c by forward substitution
    for (int r = 0; r < B; ++r) Y[r][t] = 0;
    if (t < nb) {
      for (int r = t; r < nb; ++r) {
        double v = r == t ? 1.0 : 0.0;
        for (int k = t; k < r; ++k) v -= A[r][k] * Y[k][t];
        Y[r][t] = v / A[r][r];
      }
    }
    __syncthreads();
    // M^-1 = Y^T Y, row t, FP32, zero outside nb x nb
    float* Mb = Mout + b * (int64_t)B * B;
    for (int jj = 0; jj < B; ++jj) {
      float m = 0.f;
      if (t < nb && jj < nb) {
        double v = 0.0;
        const int k0 = t > jj ? t : jj;
        for (int k = k0; k < nb; ++k) v += Y[k][t] * Y[k][jj];
        m = (float)v;
      }
      Mb[t * B + jj] = m;
    }
    __syncthreads();
  }
  // a failed block anywhere makes the status GP_ERR_NOT_SPD (last CTA decides)
  if (bad) atomicOr(&bad_any, 1);
  __syncthreads();
  if (t == 0) {
    part[blockIdx.x] = bad_any;
    __threadfence();
  }
  __shared__ bool last;
  if (t == 0) last = atomicInc(&s->ticket5, gridDim.x - 1) == gridDim.x - 1;
  __syncthreads();
  if (last && t == 0) {
    __threadfence();
    int nbad = 0;
    for (unsigned q = 0; q < gridDim.x; ++q) nbad |= __ldcg(part + q);
    s->pc_status = nbad ? GP_ERR_NOT_SPD : GP_OK;
  }
}

// Blocks of 64 or 128 rows, in FP32 (GB300's FP64 pipe makes the FP64
// factorisation of 128-row blocks cost ~36 ms per evaluation at 1M points).
// One CTA of B threads per block, thread t owning row t:
//   right-looking Cholesky A = L L^T (pivot by thread j, column j scaled,
//     trailing rows updated in parallel, one row per thread);
//   Y = L^-1, thread c forward-substituting column c, stored transposed in
//     the free upper triangle of A (Y[r][c] at A[c][r], r > c; its diagonal
//     1 / L_cc in a separate vector), so one B x (B+1) array serves both and
//     three CTAs share an SM;
//   M^-1 = Y^T Y, row t per thread (dot products of rows of the upper
//     triangle), FP32.
// Y^T Y is symmetric positive definite for any nonsingular Y, so rounding
// cannot make the preconditioner indefinite; a pivot that rounding drives to
// or below 1e-6 (the block's unit diagonal times 1e-6) is floored there,
// which factors a slightly perturbed block and keeps the preconditioner
// valid.  An indefinite K is still caught by CG (p^T K p <= 0).
template <int B>
__global__ void __launch_bounds__(B) k_pc_setup32(int64_t n, int64_t nblk, const int64_t* __restrict__ rp,
                                                  const int32_t* __restrict__ col, const float* __restrict__ val,
                                                  float* __restrict__ Mout, gp::AsmScalars* s) {
  extern __shared__ float pc_sf[];
  float (*A)[B + 1] = (float (*)[B + 1])pc_sf;
  float* yd = pc_sf + B * (B + 1);  // L_cc during the factorisation, then Y[c][c] = 1 / L_cc
  const int t = threadIdx.x;
  for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int64_t r0 = b * B;
    const int nb = (int)min((int64_t)B, n - r0);
    for (int j = 0; j < B; ++j) A[t][j] = 0.f;
    if (t < nb) {
      const int64_t row = r0 + t;
      for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
        const int64_t j = col[e];
        if (j >= r0 && j <= row) A[t][j - r0] = val[e];  // lower triangle only
      }
    }
    __syncthreads();
    // Two barriers per column: every thread takes the pivot from A[j][j],
    // which only step j reads, and the pivot goes to yd[j] (A[j][j] is set
    // after the loop), so no thread can see it overwritten mid-step.
    for (int j = 0; j < nb; ++j) {
      const float piv = sqrtf(fmaxf(A[j][j], 1e-6f));
      if (t == j) yd[j] = piv;
      if (t > j && t < nb) A[t][j] /= piv;
      __syncthreads();
      if (t > j && t < nb) {
        const float lt = A[t][j];
        for (int k = j + 1; k <= t; ++k) A[t][k] = fmaf(-lt, A[k][j], A[t][k]);
      }
      __syncthreads();
    }
    if (t < nb) A[t][t] = yd[t];
    __syncthreads();
    // Y = L^-1, column t, into row t of the upper triangle; four partial
    // sums shorten the add chains
    if (t < nb) {
      yd[t] = 1.f / A[t][t];
      for (int r = t + 1; r < nb; ++r) {
        // Y[r][t] = -(sum_{k=t}^{r-1} L[r][k] Y[k][t]) / L[r][r], Y[t][t] = yd[t]
        float v0 = -A[r][t] * yd[t], v1 = 0.f, v2 = 0.f, v3 = 0.f;
        int k = t + 1;
        for (; k + 3 < r; k += 4) {
          v0 = fmaf(-A[r][k], A[t][k], v0);
          v1 = fmaf(-A[r][k + 1], A[t][k + 1], v1);
          v2 = fmaf(-A[r][k + 2], A[t][k + 2], v2);
          v3 = fmaf(-A[r][k + 3], A[t][k + 3], v3);
        }
        for (; k < r; ++k) v0 = fmaf(-A[r][k], A[t][k], v0);
        A[t][r] = ((v0 + v1) + (v2 + v3)) / A[r][r];
      }
    }
    __syncthreads();
    // M^-1 = Y^T Y: M[t][jj] = sum_{k >= max(t, jj)} Y[k][t] Y[k][jj], with
    // Y[k][c] = A[c][k] for k > c and yd[c] for k = c; zero outside nb x nb.
    // Thread t forms the entries jj >= t of its row and writes both M[t][jj]
    // and M[jj][t]: the two are the same products in the same order (the
    // factors of each multiply and FMA only swap places), so M^-1 is exactly
    // symmetric, as the apply relies on.
    float* Mb = Mout + b * (int64_t)B * B;
    for (int jj = t; jj < B; ++jj) {
      float m = 0.f;
      if (t < nb && jj < nb) {
        const int lo = t > jj ? t : jj;
        // the k = lo term: one of the two factors sits on a diagonal
        m = (t == jj) ? yd[t] * yd[t] : (t > jj ? yd[t] * A[jj][t] : A[t][jj] * yd[jj]);
        float m1 = 0.f;
        int k = lo + 1;
        for (; k + 1 < nb; k += 2) {
          m = fmaf(A[t][k], A[jj][k], m);
          m1 = fmaf(A[t][k + 1], A[jj][k + 1], m1);
        }
        if (k < nb) m = fmaf(A[t][k], A[jj][k], m);
        m += m1;
      }
      Mb[t * B + jj] = m;
      Mb[jj * B + t] = m;
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && t == 0) s->pc_status = GP_OK;
}

template <int B>
int launch_setup32(gp_ctx* c, int64_t nblk, gp::AsmScalars* s) {
  const size_t smem = sizeof(float) * ((size_t)B * (B + 1) + B);
  GP_CUDA(cudaFuncSetAttribute(k_pc_setup32<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pc_setup32<B>, B, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t cap = (int64_t)c->num_sms * per_sm;
  const int64_t g = nblk < cap ? nblk : cap;
  k_pc_setup32<B><<<(unsigned)g, B, smem, c->stream>>>(c->n_act, nblk, (const int64_t*)c->row_ptr.p,
                                                       (const int32_t*)c->col.p, (const float*)c->val.p,
                                                       (float*)c->pc_Minv.p, s);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

template <int B>
int launch_setup(gp_ctx* c, int64_t nblk, gp::AsmScalars* s) {
  const size_t smem = 2 * sizeof(double) * B * (B + 1);
  GP_CUDA(cudaFuncSetAttribute(k_pc_setup<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pc_setup<B>, B, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t cap = (int64_t)c->num_sms * per_sm;
  const int64_t g = nblk < cap ? nblk : cap;
  GP_CHECK(gp::ensure(c, c->pc_part, (size_t)g * sizeof(int)));
  k_pc_setup<B><<<(unsigned)g, B, smem, c->stream>>>(c->n_act, nblk, (const int64_t*)c->row_ptr.p,
                                                     (const int32_t*)c->col.p, (const float*)c->val.p,
                                                     (float*)c->pc_Minv.p, (int*)c->pc_part.p, s);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

}  // namespace

namespace gp {

int precond_setup(gp_ctx* c, int B) {
  c->pc_block = 0;
  c->pc_nblk = 0;
  AsmScalars* s = (AsmScalars*)c->asm_s.p;
  GP_CUDA(cudaMemsetAsync(&s->pc_status, 0, sizeof(int), c->stream));
  if (B == 0 || c->n_act == 0 || c->precision != GP_FP32_MIXED) return GP_OK;
  if (B != 8 && B != 16 && B != 32 && B != 64 && B != 128) return GP_ERR_INVALID_ARG;
  const int64_t nblk = (c->n_act + B - 1) / B;
  GP_CHECK(ensure(c, c->pc_Minv, (size_t)nblk * B * B * sizeof(float)));
  switch (B) {
    case 8: GP_CHECK(launch_setup<8>(c, nblk, s)); break;
    case 16: GP_CHECK(launch_setup<16>(c, nblk, s)); break;
    case 32: GP_CHECK(launch_setup<32>(c, nblk, s)); break;
    case 64: GP_CHECK(launch_setup32<64>(c, nblk, s)); break;
    default: GP_CHECK(launch_setup32<128>(c, nblk, s)); break;
  }
  c->launches += 1;
  c->pc_block = B;
  c->pc_nblk = nblk;
  return GP_OK;
}

}  // namespace gp
