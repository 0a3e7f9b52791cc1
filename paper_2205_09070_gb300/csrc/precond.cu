// Block-Jacobi preconditioner of the FP32 batched CG.
//
// The active rows are in Morton / sub-cell order, so B consecutive rows are
// close in space and strongly coupled.  M = blockdiag(Khat_bb) over blocks of
// B consecutive rows; each block is factored in FP64 (one warp per block,
// Cholesky M_bb = L L^T, then M_bb^-1 = L^-T L^-1) and M^-1 is stored in FP32,
// B x B row-major per block, zero outside the block's rows for the last,
// shorter block.  Preconditioning changes only how fast CG converges: the
// solves Khat u = b it feeds are the same.
#include <math.h>

#include "gp_internal.cuh"

namespace {

constexpr int kPcMax = 32;

// One warp per diagonal block (grid-stride).  Lane i owns row i of the block.
__global__ void __launch_bounds__(32) k_pc_setup(int64_t n, int B, int64_t nblk, const int64_t* __restrict__ rp,
                                                 const int32_t* __restrict__ col, const float* __restrict__ val,
                                                 float* __restrict__ Mout, int* __restrict__ part,
                                                 gp::AsmScalars* s) {
  __shared__ double A[kPcMax][kPcMax + 1];  // block of Khat, overwritten by L (lower)
  __shared__ double Y[kPcMax][kPcMax + 1];  // L^-1 (lower)
  const int lane = threadIdx.x;
  int bad = 0;
  for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int64_t r0 = b * B;
    const int nb = (int)min((int64_t)B, n - r0);
    for (int j = 0; j < kPcMax; ++j) A[lane][j] = 0.0;
    if (lane < nb) {
      const int64_t row = r0 + lane;
      for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
        const int64_t j = col[e];
        if (j >= r0 && j < r0 + nb) A[lane][j - r0] = (double)val[e];
      }
    }
    __syncwarp();
    // Cholesky, column by column (dot-product form, lower triangle only)
    for (int j = 0; j < nb; ++j) {
      if (lane == j) {
        double d = A[j][j];
        for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
        if (!(d > 0.0)) {
          bad = 1;
          d = 1.0;
        }
        A[j][j] = sqrt(d);
      }
      __syncwarp();
      if (lane > j && lane < nb) {
        double t = A[lane][j];
        for (int k = 0; k < j; ++k) t -= A[lane][k] * A[j][k];
        A[lane][j] = t / A[j][j];
      }
      __syncwarp();
    }
    // Y = L^-1, lane c computes column c by forward substitution
    for (int r = 0; r < kPcMax; ++r) Y[r][lane] = 0.0;
    if (lane < nb) {
      for (int r = lane; r < nb; ++r) {
        double t = r == lane ? 1.0 : 0.0;
        for (int k = lane; k < r; ++k) t -= A[r][k] * Y[k][lane];
        Y[r][lane] = t / A[r][r];
      }
    }
    __syncwarp();
    // M^-1 = Y^T Y, row `lane`, FP32, zero outside nb x nb
    float* Mb = Mout + b * (int64_t)B * B;
    if (lane < B) {
      for (int jj = 0; jj < B; ++jj) {
        float m = 0.f;
        if (lane < nb && jj < nb) {
          double t = 0.0;
          const int k0 = lane > jj ? lane : jj;
          for (int k = k0; k < nb; ++k) t += Y[k][lane] * Y[k][jj];
          m = (float)t;
        }
        Mb[lane * B + jj] = m;
      }
    }
    __syncwarp();
  }
  // a failed block anywhere makes the status GP_ERR_NOT_SPD (last block decides)
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (lane == 0) {
    part[blockIdx.x] = bad;
    __threadfence();
  }
  __shared__ bool last;
  __syncwarp();
  if (lane == 0) last = atomicInc(&s->ticket5, gridDim.x - 1) == gridDim.x - 1;
  __syncwarp();
  if (last && lane == 0) {
    __threadfence();
    int nbad = 0;
    for (unsigned q = 0; q < gridDim.x; ++q) nbad |= __ldcg(part + q);
    s->pc_status = nbad ? GP_ERR_NOT_SPD : GP_OK;
  }
}

}  // namespace

namespace gp {

int precond_setup(gp_ctx* c, int B) {
  c->pc_block = 0;
  c->pc_nblk = 0;
  AsmScalars* s = (AsmScalars*)c->asm_s.p;
  GP_CUDA(cudaMemsetAsync(&s->pc_status, 0, sizeof(int), c->stream));
  if (B == 0 || c->n_act == 0 || c->precision != GP_FP32_MIXED) return GP_OK;
  if (B != 8 && B != 16 && B != 32) return GP_ERR_INVALID_ARG;
  const int64_t nblk = (c->n_act + B - 1) / B;
  GP_CHECK(ensure(c, c->pc_Minv, (size_t)nblk * B * B * sizeof(float)));
  const int64_t g = nblk < (int64_t)c->num_sms * 16 ? nblk : (int64_t)c->num_sms * 16;
  GP_CHECK(ensure(c, c->pc_part, (size_t)g * sizeof(int)));
  k_pc_setup<<<(unsigned)g, 32, 0, c->stream>>>(c->n_act, B, nblk, (const int64_t*)c->row_ptr.p,
                                                (const int32_t*)c->col.p, (const float*)c->val.p,
                                                (float*)c->pc_Minv.p, (int*)c->pc_part.p, s);
  GP_LAUNCH_CHECK();
  c->launches += 1;
  c->pc_block = B;
  c->pc_nblk = nblk;
  return GP_OK;
}

}  // namespace gp
