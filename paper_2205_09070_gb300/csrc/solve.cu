// Conjugate gradients on the Jacobi-scaled active block Khat (Sec. 2.5: K x = y
// by CG) and the stochastic Lanczos quadrature of ln|Khat| from the same CG
// iterations (the Lanczos tridiagonal of a CG run started at x0 = 0 is fixed
// by its step lengths alpha_t and direction updates beta_t).
//
// FP32_MIXED: one CG over the block [yhat, z_1 .. z_nv] (row-major, kp floats
// per row).  Per iteration t five launches:
//   A      Q = Khat P on the 8x1 block CSR (spmm.cu); per-CTA partials of p_c^T q_c
//   alpha  one block reduces A's partials in a fixed order -> alpha_c
//   B      R -= alpha Q (and Z = M^-1 R when preconditioned); partials of
//          |r_c|^2 (and r_c^T z_c)
//   beta   one block reduces B's partials -> beta_c, convergence flags, and
//          publishes the iteration-(t+1) scalars
//   C      X += alpha P_old, P = Z + beta P_old
// Scalars of iteration t live in parity slot t&1 and every kernel reads the
// iteration index from the device state, so one captured graph of launches
// serves every iteration; all reductions are deterministic.
// FP64: one single-RHS CG per column, all in FP64 (the plain comparison path),
// with its scalars finished by the last block of each kernel.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gp_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

using gpd::block_sum_partials;

__device__ inline bool last_block(unsigned* ticket) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicInc(ticket, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// alpha_c = rr_c / p_c^T q_c for columns still running (Saad, Alg. 6.18).
__device__ void finish_alpha(gp::CgState* st, const double* pq, int k, int col0, double* hist_alpha, int m_hist) {
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    double a = 0.0;
    if (!st->done[c]) {
      const double d = pq[c];
      if (!(d > 0.0) || !isfinite(d)) {
        st->status = GP_ERR_NOT_SPD;
        st->bad_col = col0 + c;
      } else {
        a = st->rr[c] / d;
        const int it = st->iter;
        if (it < m_hist) {
          hist_alpha[it * gp::kMaxCols + col0 + c] = a;
          st->steps[col0 + c] = it + 1;
        }
      }
    }
    st->alpha[c] = a;
  }
}

// beta_c = |r_new|^2 / |r|^2, convergence |r_new|^2 <= tol^2 |r_0|^2.
__device__ void finish_beta(gp::CgState* st, const double* rr_new, int k, int col0, double* hist_beta, int m_hist) {
  __shared__ int any_running;
  if (threadIdx.x == 0) any_running = 0;
  __syncthreads();
  const int it = st->iter;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    double b = 0.0;
    if (!st->done[c]) {
      const double r = rr_new[c];
      b = r / st->rr[c];
      if (it < m_hist) hist_beta[it * gp::kMaxCols + col0 + c] = b;
      st->rr[c] = r;
      if (r <= st->tol2 * st->rr0[c]) st->done[c] = 1;
      else atomicOr(&any_running, 1);
      if (!isfinite(r)) {
        st->status = GP_ERR_NOT_SPD;
        st->bad_col = col0 + c;
      }
    }
    st->beta[c] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->iter = it + 1;
    st->pending = (!any_running) || st->status != GP_OK || st->iter >= st->max_iter;
  }
}

// ---------------------------------------------------------------- FP32 batched
// Initial block B = [yhat, z_1..z_nv, 0 pad] and probe sign bits.
// Cold start (KX == nullptr): X = 0, R = P = B.  Warm start: X is kept and
// KX = Khat X was just computed, so R = P = B - Khat X (the true residual of
// the kept iterate).  Either way |r_0|^2 of the convergence test is |B|^2 per
// column, so |r| <= rtol |r_0| means the same at any starting point.
__global__ void __launch_bounds__(kThreads) k_init_f32(int64_t n, int k, int kp, const double* __restrict__ y,
                                                       const uint32_t* __restrict__ perm,
                                                       const double* __restrict__ dinv64, uint64_t seed, int nv,
                                                       float* __restrict__ X, float* __restrict__ R,
                                                       float* __restrict__ P, const float* __restrict__ KX,
                                                       uint32_t* __restrict__ zbits,
                                                       double* __restrict__ part, gp::CgState* st, double tol2,
                                                       int max_iter) {
  double acc = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = perm[p];
    const float yh = (float)(y[i] * dinv64[p]);
    acc += (double)yh * (double)yh;
    uint32_t zb[2] = {0u, 0u};
    float* xrow = X + p * kp;
    float* rrow = R + p * kp;
    float* prow = P + p * kp;
    const float* kxrow = KX ? KX + p * kp : nullptr;
    const float r0 = KX ? yh - kxrow[0] : yh;
    if (!KX) xrow[0] = 0.f;
    rrow[0] = r0;
    prow[0] = r0;
    for (int l = 0; l < nv; ++l) {
      const unsigned b = gpd::probe_bit(seed, l, (long long)i);
      zb[l >> 5] |= b << (l & 31);
      const float z = b ? -1.f : 1.f;
      const float rl = KX ? z - kxrow[1 + l] : z;
      if (!KX) xrow[1 + l] = 0.f;
      rrow[1 + l] = rl;
      prow[1 + l] = rl;
    }
    for (int c = 1 + nv; c < kp; ++c) {
      xrow[c] = 0.f;
      rrow[c] = 0.f;
      prow[c] = 0.f;
    }
    zbits[2 * p] = zb[0];
    zbits[2 * p + 1] = zb[1];
  }
  __shared__ double sh[kThreads];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sh[0];
    __threadfence();
  }
  if (last_block(&st->ticket_c)) {
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(part + b);
      st->iter = 0;
      // non-finite targets: no run (the caller gets GP_ERR_INVALID_ARG)
      st->status = isfinite(t) ? GP_OK : GP_ERR_INVALID_ARG;
      st->bad_col = isfinite(t) ? -1 : 0;
      st->max_iter = max_iter;
      st->tol2 = tol2;
      if (!isfinite(t)) t = 0.0;
      bool any = false;
      for (int c = 0; c < gp::kMaxCols; ++c) {
        const double r0 = c == 0 ? t : (c < k ? (double)n : 0.0);
        st->rr0[c] = r0;
        st->rrp[0][c] = r0;
        st->rrp[1][c] = r0;
        st->crr[0][c] = r0;
        st->crr[1][c] = r0;
        st->donep[0][c] = !(r0 > 0.0);
        st->donep[1][c] = st->donep[0][c];
        st->steps[c] = 0;
        any = any || (c < k && !st->donep[0][c]);
      }
      st->fin[0] = !any || st->status != GP_OK;
      st->fin[1] = st->fin[0];
      st->finished = st->fin[0];
    }
  }
}

__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }


constexpr int kUpdThreads = 256;
constexpr int kRedThreads = 1024;

// The per-iteration reductions spread over one CTA per column: a single CTA
// pulling all CTAs' partials (16-22 K doubles) through one SM's memory pipe
// took 12-19 us per launch, latency-bound; a column's partials, one per
// producing CTA, are summed by kColThreads threads and a fixed-order tree.
constexpr int kColThreads = 256;

// sums over b < nb of part[b * stride + col0] and (col1 >= 0) of part[b *
// stride + col1], in a fixed order, in one pass; results in thread 0
__device__ inline double2 column_sums(const double* __restrict__ part, int nb, int stride, int col0, int col1,
                                      double* red0, double* red1) {
  double a = 0.0, b2 = 0.0;
  for (int b = threadIdx.x; b < nb; b += kColThreads) {
    a += __ldcg(part + (int64_t)b * stride + col0);
    if (col1 >= 0) b2 += __ldcg(part + (int64_t)b * stride + col1);
  }
  red0[threadIdx.x] = a;
  red1[threadIdx.x] = b2;
  __syncthreads();
  for (int o = kColThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red0[threadIdx.x] += red0[threadIdx.x + o];
      red1[threadIdx.x] += red1[threadIdx.x + o];
    }
    __syncthreads();
  }
  return make_double2(red0[0], red1[0]);
}

// alpha of iteration it, CTA c for column c: alpha_c = rho_c / p_c^T q_c for
// columns still running (Saad, Alg. 6.18), p^T q from the SpMM partials; a
// non-positive or non-finite p^T q is a breakdown.  The column's state is read
// before the sum, so that its latency overlaps the sum's.
__global__ void __launch_bounds__(kColThreads) k_cg_alpha_cols(const double* __restrict__ part_pq, int npq,
                                                               int k, int kp, gp::CgState* st,
                                                               double* hist_alpha, int m_hist, gp::Group g) {
  int c = blockIdx.x;
  if (g.inst) {
    const uint32_t m = __ldg(g.map + blockIdx.x);
    const gp::GInst* I = g.inst + (m >> gp::kGroupShift);
    c = (int)(m & gp::kGroupMask);
    part_pq = I->part_a;
    npq = I->grid[gp::kGSpmm];
    st = I->st;
    hist_alpha = I->hist_alpha;
  }
  const int it = st->iter;
  if (st->fin[it & 1]) return;
  __shared__ double red0[kColThreads], red1[kColThreads];
  bool running = false;
  double rho = 0.0;
  if (threadIdx.x == 0) {
    running = c < k && !st->donep[it & 1][c];
    rho = st->rrp[it & 1][c];
  }
  const double d = column_sums(part_pq, npq, kp, c, -1, red0, red1).x;
  if (threadIdx.x == 0) {
    double a = 0.0;
    if (running) {
      if (!(d > 0.0) || !isfinite(d)) {
        st->status = GP_ERR_NOT_SPD;
        st->bad_col = c;
      } else {
        a = rho / d;
        if (it < m_hist) {
          hist_alpha[it * gp::kMaxCols + c] = a;
          st->steps[c] = it + 1;
        }
      }
    }
    st->alpha[c] = a;
  }
}

// beta and the convergence test of iteration it, CTA c for column c: rho_new
// from the partials (|r|^2, or r^T z and |r|^2 side by side in rows of 2 kp
// when preconditioned), convergence on |r|^2, the iteration-(it+1) scalars in
// parity slot (it+1)&1.  Running columns are counted in st->run_cnt; the last
// CTA to finish reads and clears the count and advances the iteration.
__global__ void __launch_bounds__(kColThreads) k_cg_beta_cols(const double* __restrict__ part, int nrr, int k,
                                                              int kp, int pc, gp::CgState* st, double* hist_beta,
                                                              int m_hist, gp::Group g) {
  int c = blockIdx.x;
  if (g.inst) {
    const uint32_t m = __ldg(g.map + blockIdx.x);
    const gp::GInst* I = g.inst + (m >> gp::kGroupShift);
    c = (int)(m & gp::kGroupMask);
    part = I->part_b;
    nrr = I->grid[pc ? gp::kGPc : gp::kGUpdR];
    st = I->st;
    hist_beta = I->hist_beta;
  }
  const int it = st->iter;
  const int cur = it & 1, nxt = (it + 1) & 1;
  if (st->fin[cur]) {
    if (c == 0 && threadIdx.x == 0) st->fin[nxt] = 1;
    return;
  }
  __shared__ double red0[kColThreads], red1[kColThreads];
  __shared__ bool last;
  const int width = pc ? 2 * kp : kp;
  bool was_done = true;
  double rrp = 0.0, crr = 0.0, lim = 0.0;
  if (threadIdx.x == 0) {
    was_done = c >= k || st->donep[cur][c];
    rrp = st->rrp[cur][c];
    crr = st->crr[cur][c];
    lim = st->tol2 * st->rr0[c];
  }
  // rho_new = r^T M^-1 r and |r|^2
  const double2 sums = column_sums(part, nrr, width, c, pc ? kp + c : -1, red0, red1);
  const double rrn = sums.x, crn = pc ? sums.y : sums.x;
  if (threadIdx.x == 0) {
    double b = 0.0;
    bool done = was_done;
    if (!was_done) {
      b = rrn / rrp;
      if (it < m_hist) hist_beta[it * gp::kMaxCols + c] = b;
      done = crn <= lim;
      if (!isfinite(rrn) || !isfinite(crn)) {
        st->status = GP_ERR_NOT_SPD;
        st->bad_col = c;
      }
    }
    st->beta[c] = b;
    st->rrp[nxt][c] = was_done ? rrp : rrn;
    st->crr[nxt][c] = was_done ? crr : crn;
    st->donep[nxt][c] = done;
    if (c < k && !done) atomicAdd(&st->run_cnt, 1u);
    __threadfence();
    last = atomicInc(&st->ticket_b, kp - 1) == (unsigned)kp - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const unsigned running = atomicExch(&st->run_cnt, 0u);
    st->iter = it + 1;
    const int f = running == 0u || __ldcg(&st->status) != GP_OK || it + 1 >= st->max_iter;
    st->fin[nxt] = f;
    st->finished = f;
  }
}

// B: R -= alpha Q with per-block partial sums of |r_c|^2.  A thread owns one
// float4 column slot (fixed, since the grid stride is a multiple of kq) and
// walks rows four at a time so that several loads are in flight; its sums
// are compensated FP32 (Dot2), the block's are combined in FP64 by a tree.
constexpr int kUpdRThreads = 1024;

__global__ void __launch_bounds__(kUpdRThreads) k_upd_r_f32(int64_t n, int kq, const float4* __restrict__ Q,
                                                            float4* __restrict__ R, double* __restrict__ part_rr,
                                                            const gp::CgState* st, gp::Group g) {
  int bx = blockIdx.x, gx = gridDim.x;
  if (g.inst) {
    const gp::GInst* I = gpd::group_cta(g, gp::kGUpdR, bx, gx);
    n = I->n;
    Q = I->Q;
    R = I->R;
    part_rr = I->part_b;
    st = I->st;
  }
  if (st->fin[st->iter & 1]) return;
  __shared__ double red[kUpdRThreads][4];
  const int ny = kUpdRThreads / kq;
  const int tx = threadIdx.x % kq, ty = threadIdx.x / kq;
  gpd::Dot2 r0, r1, r2, r3;
  if (ty < ny) {
    const float4 a = make_float4((float)st->alpha[4 * tx], (float)st->alpha[4 * tx + 1],
                                 (float)st->alpha[4 * tx + 2], (float)st->alpha[4 * tx + 3]);
    const int64_t stride = (int64_t)gx * ny;
    int64_t p = (int64_t)bx * ny + ty;
    for (; p + 3 * stride < n; p += 4 * stride) {
      float4 r[4], q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        r[u] = R[(p + u * stride) * kq + tx];
        q[u] = Q[(p + u * stride) * kq + tx];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        r[u].x = fmaf(-a.x, q[u].x, r[u].x);
        r[u].y = fmaf(-a.y, q[u].y, r[u].y);
        r[u].z = fmaf(-a.z, q[u].z, r[u].z);
        r[u].w = fmaf(-a.w, q[u].w, r[u].w);
        R[(p + u * stride) * kq + tx] = r[u];
        r0.add(r[u].x, r[u].x);
        r1.add(r[u].y, r[u].y);
        r2.add(r[u].z, r[u].z);
        r3.add(r[u].w, r[u].w);
      }
    }
    for (; p < n; p += stride) {
      float4 r = R[p * kq + tx];
      const float4 q = Q[p * kq + tx];
      r.x = fmaf(-a.x, q.x, r.x);
      r.y = fmaf(-a.y, q.y, r.y);
      r.z = fmaf(-a.z, q.z, r.z);
      r.w = fmaf(-a.w, q.w, r.w);
      R[p * kq + tx] = r;
      r0.add(r.x, r.x);
      r1.add(r.y, r.y);
      r2.add(r.z, r.z);
      r3.add(r.w, r.w);
    }
  }
  red[threadIdx.x][0] = r0.value();
  red[threadIdx.x][1] = r1.value();
  red[threadIdx.x][2] = r2.value();
  red[threadIdx.x][3] = r3.value();
  __syncthreads();
  // tree over the row index ty (same column slot tx), fixed order
  for (int h = 1; h < ny; h <<= 1) {
    if (ty < ny && (ty & (2 * h - 1)) == 0 && ty + h < ny) {
      const int o = threadIdx.x + h * kq;
#pragma unroll
      for (int q = 0; q < 4; ++q) red[threadIdx.x][q] += red[o][q];
    }
    __syncthreads();
  }
  const int kp = 4 * kq;
  if (threadIdx.x < kp) part_rr[(int64_t)bx * kp + threadIdx.x] = red[threadIdx.x / 4][threadIdx.x % 4];
}

// Start of a CG run on a caller-given right-hand-side block B (N_act x kp,
// Jacobi-scaled): X = 0, R = P = B, per-block partials of |b_c|^2 (thread per
// float4 column slot, rows strided as in k_upd_r_f32).
__global__ void __launch_bounds__(kUpdRThreads) k_rhs_init_f32(int64_t n, int kq, const float4* __restrict__ B,
                                                               float4* __restrict__ X, float4* __restrict__ R,
                                                               float4* __restrict__ P, double* __restrict__ part) {
  __shared__ double red[kUpdRThreads][4];
  const int ny = kUpdRThreads / kq;
  const int tx = threadIdx.x % kq, ty = threadIdx.x / kq;
  gpd::Dot2 b0, b1, b2, b3;
  if (ty < ny) {
    const int64_t stride = (int64_t)gridDim.x * ny;
    for (int64_t p = (int64_t)blockIdx.x * ny + ty; p < n; p += stride) {
      const float4 b = B[p * kq + tx];
      X[p * kq + tx] = make_float4(0.f, 0.f, 0.f, 0.f);
      R[p * kq + tx] = b;
      P[p * kq + tx] = b;
      b0.add(b.x, b.x);
      b1.add(b.y, b.y);
      b2.add(b.z, b.z);
      b3.add(b.w, b.w);
    }
  }
  red[threadIdx.x][0] = b0.value();
  red[threadIdx.x][1] = b1.value();
  red[threadIdx.x][2] = b2.value();
  red[threadIdx.x][3] = b3.value();
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

// The run state for k_rhs_init_f32's block: |r_0|^2 = |b_c|^2 per column
// (columns with b_c = 0 are done at once), iteration 0.
__global__ void __launch_bounds__(kRedThreads) k_rhs_state(const double* __restrict__ part, int np, int k, int kp,
                                                           gp::CgState* st, double tol2, int max_iter) {
  __shared__ double scratch[kRedThreads];
  __shared__ double sums[gp::kMaxCols];
  __shared__ int any_running;
  block_sum_partials(part, np, kp, kp, sums, scratch);
  if (threadIdx.x == 0) any_running = 0;
  __syncthreads();
  if (threadIdx.x < gp::kMaxCols) {
    const int c = threadIdx.x;
    const double r0 = c < k ? sums[c] : 0.0;
    st->rr0[c] = r0;
    st->rrp[0][c] = r0;
    st->rrp[1][c] = r0;
    st->crr[0][c] = r0;
    st->crr[1][c] = r0;
    st->steps[c] = 0;
    const bool done = !(r0 > 0.0);
    st->donep[0][c] = done;
    st->donep[1][c] = done;
    if (c < k && !done) atomicOr(&any_running, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->iter = 0;
    st->status = GP_OK;
    st->bad_col = -1;
    st->max_iter = max_iter;
    st->tol2 = tol2;
    st->fin[0] = !any_running;
    st->fin[1] = !any_running;
    st->finished = !any_running;
  }
}

// B with the block-Jacobi preconditioner M (diagonal blocks of B rows of
// Khat; B divides the tile of 32 RPL rows, so a tile holds whole blocks):
//   INIT:  Z = M^-1 R written to P (the first search direction)
//   else:  R -= alpha Q, Z = M^-1 R
// and per-block partials of rho = r^T z (columns 0..kp-1) and |r|^2
// (columns kp..2kp-1) in one row of 2 kp doubles per block.
//
// A block of 32 kq threads walks its tiles with an S-stage cp.async pipeline
// (S - 1 tiles in flight while one is computed).  Thread t copies and updates
// elements t + h 32 kq (h < RPL) of the tile-linear layout (row e / kq,
// float4 slot e % kq), so it can use its own R and Q right after its own
// copies land.  The block product runs with warp w on float4 slot w and lane
// l on rows RPL l .. RPL l + RPL - 1 (RPL = 2, or 4 for B = 128): each R row
// read from shared memory then feeds RPL rows of M^-1, whose rows are stored
// interleaved per lane (for each four columns, four of each of the lane's
// rows in turn; lane rows padded to RPL B + 4 floats, so a quarter warp's
// 16-byte reads fall in distinct banks).  Each thread's column sums stay in
// one slot across tiles and reduce with warp shuffles at the end.
constexpr int kPcLanes = 32;                       // threads per float4 slot
constexpr int kPcMaxThreads = kPcLanes * gp::kMaxCols / 4;
constexpr int pc_rows_per_lane(int B) { return B >= 128 ? 4 : 2; }
// rows per tile (B <= 32) or per block (B >= 64: one tile is one block of M^-1)
constexpr int pc_tile(int B) { return B >= 64 ? B : kPcLanes * pc_rows_per_lane(B); }
constexpr int pc_stages(int) { return 3; }
constexpr int kPcPanel = 32;  // columns of M^-1 per panel (B >= 64)

__device__ inline void cp_async16_zfill(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int nbytes = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(nbytes) : "memory");
}

size_t pc_smem_bytes(int kq, int B) {
  const size_t S = pc_stages(B);
  if (B >= 64) {
    // per stage: R and Q panels (32 rows x kq float4) and a 32-column panel of
    // M^-1 (B rows, interleaved per lane: rows padded to RPL 32 + 4 floats)
    const size_t nthr = (size_t)kPcLanes * kq;
    return S * (2 * 16 * nthr + 4 * (size_t)kPcLanes * (pc_rows_per_lane(B) * kPcPanel + 4));
  }
  const size_t tile4 = (size_t)pc_tile(B) * kq;  // float4 per R (or Q, Z) tile
  return 16 * tile4 * (2 * S + 1) + 4 * S * kPcLanes * (pc_rows_per_lane(B) * B + 4);
}

template <bool INIT, int B>
__global__ void __launch_bounds__(kPcMaxThreads) k_upd_r_pc(int64_t n, int kq,
                                                             const float4* __restrict__ Q, float4* __restrict__ R,
                                                             float4* __restrict__ Z, const float* __restrict__ Minv,
                                                             double* __restrict__ part, const gp::CgState* st, gp::Group g) {
  int bx = blockIdx.x, gx = gridDim.x;
  if (g.inst) {
    const gp::GInst* I = gpd::group_cta(g, gp::kGPc, bx, gx);
    n = I->n;
    Q = I->Q;
    R = I->R;
    Z = I->Z;
    Minv = I->Minv;
    part = I->part_b;
    st = I->st;
  }
  if (!INIT && st->fin[st->iter & 1]) return;
  constexpr int kPcStages = pc_stages(B);
  constexpr int RPL = pc_rows_per_lane(B);
  constexpr int TILE = pc_tile(B);
  extern __shared__ float4 pc_smem[];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int nthr = kPcLanes * kq;
  const int tile4 = RPL * nthr;                 // float4 per tile = TILE * kq
  constexpr int ldp = RPL * B + 4;              // floats per lane row block of M^-1
  float4* Rs = pc_smem;                         // kPcStages x tile4
  float4* Qs = Rs + kPcStages * tile4;          // kPcStages x tile4
  float4* Zs = Qs + kPcStages * tile4;          // tile4
  float* Ms = (float*)(Zs + tile4);             // kPcStages x 32 lane blocks x ldp
  const int64_t ntiles = (n + TILE - 1) / TILE;
  const int64_t nrows_pc = (n + B - 1) / B * B;  // rows covered by stored blocks
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!INIT) {
    const int q = t % kq;  // also the slot of elements t + h nthr (nthr is a multiple of kq)
    a = make_float4((float)st->alpha[4 * q], (float)st->alpha[4 * q + 1], (float)st->alpha[4 * q + 2],
                    (float)st->alpha[4 * q + 3]);
  }
  auto issue = [&](int64_t tile, int s) {
    if (tile < ntiles) {
      const int64_t r0 = tile * TILE;
#pragma unroll
      for (int h = 0; h < RPL; ++h) {
        const int e = t + h * nthr;
        const bool ok = r0 + e / kq < n;
        const int64_t src = ok ? r0 * kq + e : 0;
        cp_async16_zfill(Rs + s * tile4 + e, R + src, ok);
        if (!INIT) cp_async16_zfill(Qs + s * tile4 + e, Q + src, ok);
      }
      constexpr int c4n = B / 4;
      for (int e = t; e < TILE * c4n; e += nthr) {
        const int r = e / c4n, c4 = e - r * c4n;
        const bool okm = r0 + r < nrows_pc;
        const float* srcm = Minv + (okm ? (r0 + r) * B + 4 * c4 : 0);
        cp_async16_zfill(Ms + (s * kPcLanes + r / RPL) * ldp + 4 * RPL * c4 + 4 * (r % RPL), srcm, okm);
      }
    }
    cp_async_commit();  // empty groups past the end keep the group count uniform
  };
  gpd::Dot2 rz[4], rr[4];
  const int kb = ((RPL * lane) / B) * B;  // first tile row of this lane's block
  int64_t tile = bx;
#pragma unroll
  for (int q = 0; q < kPcStages - 1; ++q) issue(tile + q * (int64_t)gx, q);
  for (int i = 0; tile < ntiles; ++i, tile += gx) {
    const int s = i % kPcStages;
    issue(tile + (kPcStages - 1) * (int64_t)gx, (i + kPcStages - 1) % kPcStages);
    cp_async_wait<kPcStages - 1>();  // this thread's copies of tile i have landed
    const int64_t r0 = tile * TILE;
    if (!INIT) {
#pragma unroll
      for (int h = 0; h < RPL; ++h) {
        const int e = t + h * nthr;
        float4 v = Rs[s * tile4 + e];
        const float4 qv = Qs[s * tile4 + e];
        v.x = fmaf(-a.x, qv.x, v.x);
        v.y = fmaf(-a.y, qv.y, v.y);
        v.z = fmaf(-a.z, qv.z, v.z);
        v.w = fmaf(-a.w, qv.w, v.w);
        Rs[s * tile4 + e] = v;
        if (r0 + e / kq < n) R[r0 * kq + e] = v;
      }
    }
    __syncthreads();
    {
      const float4* Rt = Rs + s * tile4;
      const float* mrow = Ms + (s * kPcLanes + lane) * ldp;
      float2 zlo[RPL], zhi[RPL];
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        zlo[u] = make_float2(0.f, 0.f);
        zhi[u] = make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < B; k += 4) {
        float4 m[RPL];  // rows RPL l + u, columns k..k+3
#pragma unroll
        for (int u = 0; u < RPL; ++u) m[u] = *(const float4*)(mrow + RPL * k + 4 * u);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float4 x = Rt[(kb + k + c) * kq + w];
          const float2 xlo = make_float2(x.x, x.y), xhi = make_float2(x.z, x.w);
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const float mc = c == 0 ? m[u].x : c == 1 ? m[u].y : c == 2 ? m[u].z : m[u].w;
            const float2 a2 = make_float2(mc, mc);
            zlo[u] = __ffma2_rn(a2, xlo, zlo[u]);
            zhi[u] = __ffma2_rn(a2, xhi, zhi[u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        const float4 rv = Rt[(RPL * lane + u) * kq + w];
        const float4 z = make_float4(zlo[u].x, zlo[u].y, zhi[u].x, zhi[u].y);
        Zs[(RPL * lane + u) * kq + w] = z;
        rz[0].add(rv.x, z.x);
        rz[1].add(rv.y, z.y);
        rz[2].add(rv.z, z.z);
        rz[3].add(rv.w, z.w);
        rr[0].add(rv.x, rv.x);
        rr[1].add(rv.y, rv.y);
        rr[2].add(rv.z, rv.z);
        rr[3].add(rv.w, rv.w);
      }
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < RPL; ++h) {
      const int e = t + h * nthr;
      if (r0 + e / kq < n) Z[r0 * kq + e] = Zs[e];
    }
  }
  cp_async_wait<0>();
  // rows beyond n were filled with zeros, so they added nothing above
  double v[8];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = rz[j].value();
    v[4 + j] = rr[j].value();
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(kFull, v[j], o);
  if (lane == 0) {
    const int kp = 4 * kq;
    double* prow = part + (int64_t)bx * 2 * kp;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      prow[4 * w + j] = v[j];
      prow[kp + 4 * w + j] = v[4 + j];
    }
  }
}

// The same update for B = 64 or 128, with M^-1 streamed in panels of 32
// columns: a block of rows r0 .. r0 + B - 1 (one block of M^-1) is taken in
// B / 32 panels, panel q bringing rows r0 + 32q .. r0 + 32q + 31 of R and Q
// and columns 32q .. 32q + 31 of the block's M^-1.  Thread t updates element
// t of the panel (R -= alpha Q); then lane l adds the panel's share
//   z[RPL l + u] += sum_{k < 32} M^-1[RPL l + u][32q + k] R[32q + k]
// for its RPL = B / 32 rows and warp w's float4 slot, so Z stays in registers
// across the block's panels and a stage holds only 26 KB (3 stages, two CTAs
// per SM) where a whole 128 x 128 block of M^-1 would take 64 KB.  The panel
// stream runs across the CTA's blocks without a break, one barrier per panel.
template <bool INIT, int B>
__global__ void __launch_bounds__(kPcMaxThreads) k_upd_r_pcp(int64_t n, int kq,
                                                              const float4* __restrict__ Q, float4* __restrict__ R,
                                                              float4* __restrict__ Z, const float* __restrict__ Minv,
                                                              double* __restrict__ part, const gp::CgState* st, gp::Group g) {
  int bx = blockIdx.x, gx = gridDim.x;
  if (g.inst) {
    const gp::GInst* I = gpd::group_cta(g, gp::kGPc, bx, gx);
    n = I->n;
    Q = I->Q;
    R = I->R;
    Z = I->Z;
    Minv = I->Minv;
    part = I->part_b;
    st = I->st;
  }
  if (!INIT && st->fin[st->iter & 1]) return;
  constexpr int S = pc_stages(B);
  constexpr int RPL = B / kPcLanes;  // rows per lane
  constexpr int NPB = B / kPcPanel;  // panels per block
  constexpr int ldm = RPL * kPcPanel + 4;
  extern __shared__ float4 pc_smem[];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int nthr = kPcLanes * kq;  // float4 per R (or Q) panel
  float4* Rs = pc_smem;            // S x nthr
  float4* Qs = Rs + S * nthr;      // S x nthr
  float* Ms = (float*)(Qs + S * nthr);  // S x 32 lane groups x ldm
  const int64_t nblk = (n + B - 1) / B;
  const int64_t mine = bx < nblk ? (nblk - 1 - bx) / gx + 1 : 0;
  const int64_t npan = mine * NPB;
  const int64_t nrows_pc = nblk * B;
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!INIT) {
    const int q = t % kq;
    a = make_float4((float)st->alpha[4 * q], (float)st->alpha[4 * q + 1], (float)st->alpha[4 * q + 2],
                    (float)st->alpha[4 * q + 3]);
  }
  auto issue = [&](int64_t pi, int s) {
    if (pi < npan) {
      const int64_t blk = bx + (pi / NPB) * gx;
      const int q = (int)(pi % NPB);
      const int64_t r0 = blk * B + kPcPanel * q;  // first row of the panel
      const bool ok = r0 + t / kq < n;
      const int64_t src = ok ? r0 * kq + t : 0;
      cp_async16_zfill(Rs + s * nthr + t, R + src, ok);
      if (!INIT) cp_async16_zfill(Qs + s * nthr + t, Q + src, ok);
      for (int e = t; e < B * (kPcPanel / 4); e += nthr) {
        const int r = e / (kPcPanel / 4), c4 = e - r * (kPcPanel / 4);
        const int64_t grow = blk * B + r;
        const bool okm = grow < nrows_pc;
        const float* srcm = Minv + (okm ? grow * B + kPcPanel * q + 4 * c4 : 0);
        cp_async16_zfill(Ms + (s * kPcLanes + r / RPL) * ldm + 4 * RPL * c4 + 4 * (r % RPL), srcm, okm);
      }
    }
    cp_async_commit();
  };
  gpd::Dot2 rz[4], rr[4];
  float2 zlo[RPL], zhi[RPL];
  float4 rv[RPL];
#pragma unroll
  for (int q = 0; q < S - 1; ++q) issue(q, q);
  for (int64_t pi = 0; pi < npan; ++pi) {
    const int s = (int)(pi % S);
    cp_async_wait<S - 2>();  // this thread's copies of panel pi have landed
    const int q = (int)(pi % NPB);
    const int64_t blk = bx + (pi / NPB) * gx;
    const int64_t r0 = blk * B + kPcPanel * q;
    if (q == 0) {
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        zlo[u] = make_float2(0.f, 0.f);
        zhi[u] = make_float2(0.f, 0.f);
      }
    }
    if (!INIT) {
      float4 v = Rs[s * nthr + t];
      const float4 qv = Qs[s * nthr + t];
      v.x = fmaf(-a.x, qv.x, v.x);
      v.y = fmaf(-a.y, qv.y, v.y);
      v.z = fmaf(-a.z, qv.z, v.z);
      v.w = fmaf(-a.w, qv.w, v.w);
      Rs[s * nthr + t] = v;
      if (r0 + t / kq < n) R[r0 * kq + t] = v;
    }
    // one barrier per panel: panel pi's copies and updates are visible to all
    // threads, and every thread has finished panel pi-1, whose stage the next
    // copies refill (S - 1 panels stay in flight while pi is computed)
    __syncthreads();
    issue(pi + S - 1, (int)((pi + S - 1) % S));
    const float4* Rt = Rs + s * nthr;
    // the lane's own rows RPL l .. RPL l + RPL - 1 of the block lie in panel (RPL l) / 32
    if ((RPL * lane) / kPcPanel == q) {
#pragma unroll
      for (int u = 0; u < RPL; ++u) rv[u] = Rt[((RPL * lane + u) % kPcPanel) * kq + w];
    }
    const float* mrow = Ms + (s * kPcLanes + lane) * ldm;
#pragma unroll
    for (int k = 0; k < kPcPanel; k += 4) {
      float4 m[RPL];
#pragma unroll
      for (int u = 0; u < RPL; ++u) m[u] = *(const float4*)(mrow + RPL * k + 4 * u);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float4 x = Rt[(k + c) * kq + w];
        const float2 xlo = make_float2(x.x, x.y), xhi = make_float2(x.z, x.w);
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const float mc = c == 0 ? m[u].x : c == 1 ? m[u].y : c == 2 ? m[u].z : m[u].w;
          const float2 a2 = make_float2(mc, mc);
          zlo[u] = __ffma2_rn(a2, xlo, zlo[u]);
          zhi[u] = __ffma2_rn(a2, xhi, zhi[u]);
        }
      }
    }
    if (q == NPB - 1) {
      // the block's Z rows of this lane are complete: write them, add r.z, r.r
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        const int64_t row = blk * B + RPL * lane + u;
        const float4 z = make_float4(zlo[u].x, zlo[u].y, zhi[u].x, zhi[u].y);
        if (row < n) Z[row * kq + w] = z;
        rz[0].add(rv[u].x, z.x);
        rz[1].add(rv[u].y, z.y);
        rz[2].add(rv[u].z, z.z);
        rz[3].add(rv[u].w, z.w);
        rr[0].add(rv[u].x, rv[u].x);
        rr[1].add(rv[u].y, rv[u].y);
        rr[2].add(rv[u].z, rv[u].z);
        rr[3].add(rv[u].w, rv[u].w);
      }
    }
  }
  cp_async_wait<0>();
  // rows beyond n were filled with zeros, so they added nothing above
  double v[8];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = rz[j].value();
    v[4 + j] = rr[j].value();
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(kFull, v[j], o);
  if (lane == 0) {
    const int kp = 4 * kq;
    double* prow = part + (int64_t)bx * 2 * kp;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      prow[4 * w + j] = v[j];
      prow[kp + 4 * w + j] = v[4 + j];
    }
  }
}

// B = 128 with a two-dimensional split inside each warp: warp w keeps float4
// slot w, and its lanes form 16 row groups (8 rows each) x 2 k groups, lane
// (g, h) accumulating
//   z[8 g + i] += M^-1[8 g + i][k] R[k],  k = 32q + 2kk + h, kk < 16,
// over the block's panels.  Per k a lane reads 8 entries of M^-1 (row k of
// the panel: M^-1 is exactly symmetric) and one float4 of R for 32 FMAs, so
// a warp gets 1024 FMAs from 12 shared wavefronts where the one-dimensional
// split (4 rows per lane, all 128 k) got 512 from 8; 8 rows keep the
// kernel within the 96 registers that two CTAs of 288 threads per SM allow.
// The panel row pitch of 132 floats and the interleaved k keep the loads free
// of bank conflicts.  At the end of a block the two k-group partial sums of
// each row are combined by a shuffle reduce-scatter (each lane keeps 4 of its
// 8 rows).
template <bool INIT>
__global__ void __launch_bounds__(kPcMaxThreads) k_upd_r_pcq(int64_t n, int kq,
                                                                 const float4* __restrict__ Q,
                                                                 float4* __restrict__ R, float4* __restrict__ Z,
                                                                 const float* __restrict__ Minv,
                                                                 double* __restrict__ part,
                                                                 const gp::CgState* st, gp::Group g) {
  int bx = blockIdx.x, gx = gridDim.x;
  if (g.inst) {
    const gp::GInst* I = gpd::group_cta(g, gp::kGPc, bx, gx);
    n = I->n;
    Q = I->Q;
    R = I->R;
    Z = I->Z;
    Minv = I->Minv;
    part = I->part_b;
    st = I->st;
  }
  if (!INIT && st->fin[st->iter & 1]) return;
  constexpr int B = 128;
  constexpr int S = pc_stages(B);
  constexpr int NPB = B / kPcPanel;  // panels per block
  constexpr int ldm = B + 4;         // panel row pitch (floats)
  extern __shared__ float4 pc_smem[];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int rg = lane >> 1, kg = lane & 1;
  const int nthr = kPcLanes * kq;        // float4 per R (or Q) panel
  float4* Rs = pc_smem;                  // S x nthr
  float4* Qs = Rs + S * nthr;            // S x nthr
  float* Ms = (float*)(Qs + S * nthr);   // S x 32 x ldm: rows of M^-1
  const int64_t nblk = (n + B - 1) / B;
  const int64_t mine = bx < nblk ? (nblk - 1 - bx) / gx + 1 : 0;
  const int64_t npan = mine * NPB;
  const int64_t nrows_pc = nblk * B;
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!INIT) {
    const int q = t % kq;
    a = make_float4((float)st->alpha[4 * q], (float)st->alpha[4 * q + 1], (float)st->alpha[4 * q + 2],
                    (float)st->alpha[4 * q + 3]);
  }
  auto issue = [&](int64_t pi, int s) {
    if (pi < npan) {
      const int64_t blk = bx + (pi / NPB) * gx;
      const int q = (int)(pi % NPB);
      const int64_t r0 = blk * B + kPcPanel * q;  // first row of the panel
      const bool ok = r0 + t / kq < n;
      const int64_t src = ok ? r0 * kq + t : 0;
      cp_async16_zfill(Rs + s * nthr + t, R + src, ok);
      if (!INIT) cp_async16_zfill(Qs + s * nthr + t, Q + src, ok);
      for (int e = t; e < kPcPanel * (B / 4); e += nthr) {
        const int kr = e / (B / 4), c4 = e - kr * (B / 4);
        const int64_t grow = r0 + kr;  // row of the stacked blocks of M^-1
        const bool okm = grow < nrows_pc;
        const float* srcm = Minv + (okm ? grow * B + 4 * c4 : 0);
        cp_async16_zfill(Ms + (s * kPcPanel + kr) * ldm + 4 * c4, srcm, okm);
      }
    }
    cp_async_commit();
  };
  gpd::Dot2 rz[4], rr[4];
  float2 acc[8][2];  // acc[i] = z[8 rg + i], columns (x, y) and (z, w) of slot w
  float4 rv[4];
  // the rows this lane holds after the reduce-scatter
  const int myrow0 = 8 * rg + 4 * kg;
#pragma unroll
  for (int q = 0; q < S - 1; ++q) issue(q, q);
  for (int64_t pi = 0; pi < npan; ++pi) {
    const int s = (int)(pi % S);
    cp_async_wait<S - 2>();  // this thread's copies of panel pi have landed
    const int q = (int)(pi % NPB);
    const int64_t blk = bx + (pi / NPB) * gx;
    const int64_t r0 = blk * B + kPcPanel * q;
    if (q == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
    }
    if (!INIT) {
      float4 v = Rs[s * nthr + t];
      const float4 qv = Qs[s * nthr + t];
      v.x = fmaf(-a.x, qv.x, v.x);
      v.y = fmaf(-a.y, qv.y, v.y);
      v.z = fmaf(-a.z, qv.z, v.z);
      v.w = fmaf(-a.w, qv.w, v.w);
      Rs[s * nthr + t] = v;
      if (r0 + t / kq < n) R[r0 * kq + t] = v;
    }
    // one barrier per panel (as in k_upd_r_pcp)
    __syncthreads();
    issue(pi + S - 1, (int)((pi + S - 1) % S));
    const float4* Rt = Rs + s * nthr;
    if (myrow0 / kPcPanel == q) {
#pragma unroll
      for (int u = 0; u < 4; ++u) rv[u] = Rt[((myrow0 + u) % kPcPanel) * kq + w];
    }
    const float* mrow = Ms + s * kPcPanel * ldm + 8 * rg;
#pragma unroll 8
    for (int kk = 0; kk < kPcPanel / 2; ++kk) {
      const int k = 2 * kk + kg;
      const float4* mk = (const float4*)(mrow + k * ldm);
      const float4 x = Rt[k * kq + w];
      const float2 xlo = make_float2(x.x, x.y), xhi = make_float2(x.z, x.w);
#pragma unroll
      for (int c4 = 0; c4 < 2; ++c4) {
        const float4 m = mk[c4];
        const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 m2v = make_float2(mv[i], mv[i]);
          acc[4 * c4 + i][0] = __ffma2_rn(m2v, xlo, acc[4 * c4 + i][0]);
          acc[4 * c4 + i][1] = __ffma2_rn(m2v, xhi, acc[4 * c4 + i][1]);
        }
      }
    }
    if (q == NPB - 1) {
      // reduce-scatter over the two k groups: a lane keeps rows 4 kg .. + 3 of its 8
      const bool b0 = kg;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float2 zc[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float2 lo = acc[u][c], hi = acc[u + 4][c];
          const float2 send = b0 ? lo : hi, keep = b0 ? hi : lo;
          zc[c] = make_float2(keep.x + __shfl_xor_sync(kFull, send.x, 1),
                              keep.y + __shfl_xor_sync(kFull, send.y, 1));
        }
        const float4 z = make_float4(zc[0].x, zc[0].y, zc[1].x, zc[1].y);
        const int64_t row = blk * B + myrow0 + u;
        if (row < n) Z[row * kq + w] = z;
        rz[0].add(rv[u].x, z.x);
        rz[1].add(rv[u].y, z.y);
        rz[2].add(rv[u].z, z.z);
        rz[3].add(rv[u].w, z.w);
        rr[0].add(rv[u].x, rv[u].x);
        rr[1].add(rv[u].y, rv[u].y);
        rr[2].add(rv[u].z, rv[u].z);
        rr[3].add(rv[u].w, rv[u].w);
      }
    }
  }
  cp_async_wait<0>();
  // rows beyond n were filled with zeros, so they added nothing above
  double v[8];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = rz[j].value();
    v[4 + j] = rr[j].value();
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(kFull, v[j], o);
  if (lane == 0) {
    const int kp = 4 * kq;
    double* prow = part + (int64_t)bx * 2 * kp;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      prow[4 * w + j] = v[j];
      prow[kp + 4 * w + j] = v[4 + j];
    }
  }
}

typedef void (*UpdPcFn)(int64_t, int, const float4*, float4*, float4*, const float*, double*, const gp::CgState*,
                        gp::Group);

template <bool INIT>
UpdPcFn upd_pc_fn(int B) {
  switch (B) {
    case 8: return k_upd_r_pc<INIT, 8>;
    case 16: return k_upd_r_pc<INIT, 16>;
    case 32: return k_upd_r_pc<INIT, 32>;
    case 64: return k_upd_r_pcp<INIT, 64>;
    case 128: return k_upd_r_pcq<INIT>;
    default: return nullptr;
  }
}

// Preconditioned start: rho_0 = r^T M^-1 r drives alpha / beta; a column whose
// starting residual already meets |r| <= rtol |B| is done.
__global__ void __launch_bounds__(kRedThreads) k_pc_state(const double* __restrict__ part, int np, int k, int kp,
                                                          gp::CgState* st) {
  __shared__ double scratch[kRedThreads];
  __shared__ double sums[2 * gp::kMaxCols];
  __shared__ int any_running;
  block_sum_partials(part, np, 2 * kp, 2 * kp, sums, scratch);
  if (threadIdx.x == 0) any_running = 0;
  __syncthreads();
  if (threadIdx.x < gp::kMaxCols) {
    const int c = threadIdx.x;
    const double p0 = c < k ? sums[c] : 0.0;
    const double r0 = c < k ? sums[kp + c] : 0.0;
    // rr0 stays |B|^2 from the init (the right-hand side, whatever the start)
    st->crr[0][c] = r0;
    st->crr[1][c] = r0;
    st->rrp[0][c] = p0;
    st->rrp[1][c] = p0;
    const bool done = !(r0 > 0.0) || !(p0 > 0.0) || r0 <= st->tol2 * st->rr0[c];
    st->donep[0][c] = done;
    st->donep[1][c] = done;
    if (c < k && !done) atomicOr(&any_running, 1);
    if (c < k && (!isfinite(r0) || !isfinite(p0))) {
      st->status = GP_ERR_NOT_SPD;
      st->bad_col = c;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int f = !any_running || st->status != GP_OK;
    st->fin[0] = f;
    st->fin[1] = f;
    st->finished = f;
  }
}

// C: X += alpha P_old, P = Z + beta P_old with Z = M^-1 R (Z = R without a
// preconditioner); runs for iteration it unless the run had already finished.
__global__ void __launch_bounds__(kUpdThreads) k_upd_xp_f32(int64_t n, int kq, float4* __restrict__ X,
                                                            const float4* __restrict__ R, float4* __restrict__ P,
                                                            const gp::CgState* st, gp::Group g) {
  int bx = blockIdx.x, gx = gridDim.x;
  if (g.inst) {
    const gp::GInst* I = gpd::group_cta(g, gp::kGUpd, bx, gx);
    n = I->n;
    X = I->X;
    R = I->D;
    P = I->P;
    st = I->st;
  }
  // beta has already advanced the counter for this iteration (or, when the
  // run had finished, marked the parity slot of it - 1 finished as well)
  if (st->fin[(st->iter - 1) & 1]) return;
  const int ny = kUpdThreads / kq;
  const int tx = threadIdx.x % kq, ty = threadIdx.x / kq;
  if (ty >= ny) return;
  const float4 a = make_float4((float)st->alpha[4 * tx], (float)st->alpha[4 * tx + 1], (float)st->alpha[4 * tx + 2],
                               (float)st->alpha[4 * tx + 3]);
  const float4 b = make_float4((float)st->beta[4 * tx], (float)st->beta[4 * tx + 1], (float)st->beta[4 * tx + 2],
                               (float)st->beta[4 * tx + 3]);
  const int64_t stride = (int64_t)gx * ny;
  int64_t p = (int64_t)bx * ny + ty;
  for (; p + stride < n; p += 2 * stride) {
    float4 po[2], r[2], x[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t o = (p + u * stride) * kq + tx;
      po[u] = P[o];
      r[u] = R[o];
      x[u] = X[o];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t o = (p + u * stride) * kq + tx;
      x[u].x = fmaf(a.x, po[u].x, x[u].x);
      x[u].y = fmaf(a.y, po[u].y, x[u].y);
      x[u].z = fmaf(a.z, po[u].z, x[u].z);
      x[u].w = fmaf(a.w, po[u].w, x[u].w);
      X[o] = x[u];
      P[o] = make_float4(fmaf(b.x, po[u].x, r[u].x), fmaf(b.y, po[u].y, r[u].y), fmaf(b.z, po[u].z, r[u].z),
                         fmaf(b.w, po[u].w, r[u].w));
    }
  }
  for (; p < n; p += stride) {
    const int64_t o = p * kq + tx;
    const float4 po = P[o];
    const float4 r = R[o];
    float4 x = X[o];
    x.x = fmaf(a.x, po.x, x.x);
    x.y = fmaf(a.y, po.y, x.y);
    x.z = fmaf(a.z, po.z, x.z);
    x.w = fmaf(a.w, po.w, x.w);
    X[o] = x;
    P[o] = make_float4(fmaf(b.x, po.x, r.x), fmaf(b.y, po.y, r.y), fmaf(b.z, po.z, r.z), fmaf(b.w, po.w, r.w));
  }
}

// ---------------------------------------------------------------- FP64 single RHS
__global__ void __launch_bounds__(kThreads) k_init_f64(int64_t n, int col0, int nv, const double* __restrict__ y,
                                                       const uint32_t* __restrict__ perm,
                                                       const double* __restrict__ dinv64,
                                                       const double* __restrict__ rhs, uint64_t seed,
                                                       double* __restrict__ X, double* __restrict__ R,
                                                       double* __restrict__ P, uint32_t* __restrict__ zbits,
                                                       double* __restrict__ part, gp::CgState* st, double tol2,
                                                       int max_iter) {
  double acc = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = perm[p];
    double v;
    if (rhs) {
      v = rhs[(int64_t)col0 * n + p];
    } else if (col0 == 0) {
      v = y[i] * dinv64[p];
      uint32_t zb[2] = {0u, 0u};
      for (int l = 0; l < nv; ++l) zb[l >> 5] |= gpd::probe_bit(seed, l, (long long)i) << (l & 31);
      zbits[2 * p] = zb[0];
      zbits[2 * p + 1] = zb[1];
    } else {
      v = gpd::probe_bit(seed, col0 - 1, (long long)i) ? -1.0 : 1.0;
    }
    X[p] = 0.0;
    R[p] = v;
    P[p] = v;
    acc += v * v;
  }
  __shared__ double sh[kThreads];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
  if (last_block(&st->ticket_c)) {
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(part + b);
      st->iter = 0;
      // non-finite targets (or right-hand side): no run, GP_ERR_INVALID_ARG
      st->status = isfinite(t) ? GP_OK : GP_ERR_INVALID_ARG;
      st->bad_col = isfinite(t) ? -1 : col0;
      if (!isfinite(t)) t = 0.0;
      st->max_iter = max_iter;
      st->tol2 = tol2;
      st->rr0[0] = t;
      st->rr[0] = t;
      st->alpha[0] = 0.0;
      st->beta[0] = 0.0;
      st->done[0] = !(t > 0.0);
      st->steps[col0] = 0;
      st->pending = st->done[0];
      st->finished = st->done[0];
    }
  }
}

// A (FP64): q = Khat p, one warp per row, lanes over the row's nonzeros.
__global__ void __launch_bounds__(kThreads) k_spmv_f64(int64_t n, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ col,
                                                       const double* __restrict__ val, const double* __restrict__ P,
                                                       double* __restrict__ Q, double* __restrict__ part,
                                                       gp::CgState* st, int col0, double* hist_alpha, int m_hist) {
  if (st->finished) return;
  __shared__ double sh[kWarps];
  __shared__ double tot[1];
  __shared__ double scratch[kThreads];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double pq = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * kWarps + w; p < n; p += (int64_t)gridDim.x * kWarps) {
    double q = 0.0;
    for (int64_t e = rp[p] + lane; e < rp[p + 1]; e += 32) q = fma(__ldg(val + e), __ldg(P + __ldg(col + e)), q);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(kFull, q, o);
    if (lane == 0) {
      Q[p] = q;
      pq += P[p] * q;
    }
  }
  if (lane == 0) sh[w] = pq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int ww = 0; ww < kWarps; ++ww) t += sh[ww];
    part[blockIdx.x] = t;
  }
  if (last_block(&st->ticket_a)) {
    block_sum_partials(part, gridDim.x, 1, 1, tot, scratch);
    finish_alpha(st, tot, 1, col0, hist_alpha, m_hist);
  }
}

__global__ void __launch_bounds__(kThreads) k_upd_r_f64(int64_t n, const double* __restrict__ Q,
                                                        double* __restrict__ R, double* __restrict__ part,
                                                        gp::CgState* st, int col0, double* hist_beta, int m_hist) {
  if (st->finished) return;
  __shared__ double sh[kThreads];
  __shared__ double tot[1];
  const double a = st->alpha[0];
  double acc = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double r = fma(-a, Q[p], R[p]);
    R[p] = r;
    acc += r * r;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
  if (last_block(&st->ticket_b)) {
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(part + b);
      tot[0] = t;
    }
    __syncthreads();
    finish_beta(st, tot, 1, col0, hist_beta, m_hist);
  }
}

__global__ void __launch_bounds__(kThreads) k_upd_xp_f64(int64_t n, double* __restrict__ X,
                                                         const double* __restrict__ R, double* __restrict__ P,
                                                         gp::CgState* st) {
  if (st->finished) return;
  const double a = st->alpha[0], b = st->beta[0];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double po = P[p];
    X[p] = fma(a, po, X[p]);
    P[p] = fma(b, po, R[p]);
  }
  if (last_block(&st->ticket_c)) {
    if (threadIdx.x == 0) st->finished = st->pending;
  }
}

// ---------------------------------------------------------------- LML pieces
// Inactive rows (outside every bump): K_ii = sigma_n^2 only; sum y_i^2 there.
__global__ void __launch_bounds__(kThreads) k_inactive(int64_t n, const double* __restrict__ y,
                                                       const uint32_t* __restrict__ mask0, double* part,
                                                       gp::AsmScalars* s) {
  double acc = 0.0;
  long long cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (mask0[i] == 0u) {
      acc += y[i] * y[i];
      ++cnt;
    }
  }
  __shared__ double sh[kThreads];
  __shared__ long long shc[kThreads];
  sh[threadIdx.x] = acc;
  shc[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[threadIdx.x] += sh[threadIdx.x + o];
      shc[threadIdx.x] += shc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sh[0];
    ((long long*)part)[2 * blockIdx.x + 1] = shc[0];
  }
  if (last_block(&s->ticket2)) {
    if (threadIdx.x == 0) {
      double t = 0.0;
      long long c = 0;
      for (unsigned b = 0; b < gridDim.x; ++b) {
        t += __ldcg(part + 2 * b);
        c += __ldcg((const long long*)part + 2 * b + 1);
      }
      s->inact_y2 = t;
      s->n_inactive = c;
    }
  }
}

// y_act^T K_act^-1 y_act = yhat^T alphahat with yhat = D^-1/2 y.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_quad(int64_t n, const double* __restrict__ y,
                                                   const uint32_t* __restrict__ perm,
                                                   const double* __restrict__ dinv64, const T* __restrict__ X,
                                                   int64_t ld, double* part, gp::AsmScalars* s) {
  double acc = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    acc += y[perm[p]] * dinv64[p] * (double)X[p * ld];
  __shared__ double sh[kThreads];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
  if (last_block(&s->ticket3)) {
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(part + b);
      s->quad_form = t;
    }
  }
}

// Eigenvalues and first eigenvector components of the symmetric tridiagonal
// T (diagonal d[0..m), off-diagonal e[0..m-1)) by the implicit QL method with
// Wilkinson-type shifts (Wilkinson & Reinsch; Golub & Van Loan Sec. 8.3),
// accumulating only the first row z of the eigenvector matrix (Golub & Welsch).
// Returns false if it fails to converge.
__device__ bool tridiag_ql(double* d, double* e, double* z, int m) {
  for (int i = 0; i < m; ++i) z[i] = i == 0 ? 1.0 : 0.0;
  if (m > 0) e[m - 1] = 0.0;
  for (int l = 0; l < m; ++l) {
    int iter = 0;
    for (;;) {
      int mm = l;
      for (; mm < m - 1; ++mm) {
        const double dd = fabs(d[mm]) + fabs(d[mm + 1]);
        if (fabs(e[mm]) <= 1e-16 * dd) break;
      }
      if (mm == l) break;
      if (++iter > 60) return false;
      // shift from the leading 2x2 block
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[mm] - d[l] + e[l] / (g + (g >= 0.0 ? fabs(r) : -fabs(r)));
      double s = 1.0, c = 1.0, p = 0.0;
      int i = mm - 1;
      bool deflated = false;
      for (; i >= l; --i) {
        const double f = s * e[i];
        const double b = c * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[mm] = 0.0;
          deflated = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        const double zf = z[i + 1];
        z[i + 1] = s * z[i] + c * zf;
        z[i] = c * z[i] - s * zf;
      }
      if (deflated) continue;
      d[l] -= p;
      e[l] = g;
      e[mm] = 0.0;
    }
  }
  return true;
}

// One block per probe (the eigen-solve is serial FP64 work, so each probe
// gets an SM's FP64 units of its own): Lanczos T from the CG coefficients
// of column 1+l (Saad, Sec. 6.7.3): T_tt = 1/alpha_t + beta_{t-1}/alpha_{t-1},
// T_t,t+1 = sqrt(beta_t)/alpha_t; Gamma_l = |z|^2 sum_k tau_k^2 ln theta_k.
// The last block to finish forms the mean and variance over probes.
// The kernel runs on a side stream under the preconditioned CG, so it is held
// to 32 registers: a block of 32 threads then takes exactly the 1024
// registers that three CTAs of the wide SpMM (128 threads x 168) leave free
// on an SM, and the SpMM keeps its single wave of 3 CTAs on every SM.
__global__ void __maxnreg__(32) k_slq(int nv, int64_t n_act, const double* __restrict__ ha, const double* __restrict__ hb,
                      const int* __restrict__ steps, double* gam, gp::AsmScalars* s) {
  const int l = blockIdx.x;
  if (threadIdx.x == 0) {
    const int c = 1 + l;
    const int m = steps[c];
    double d[gp::kMaxLanczos], e[gp::kMaxLanczos], z[gp::kMaxLanczos];
    for (int t = 0; t < m; ++t) {
      const double at = ha[t * gp::kMaxCols + c];
      d[t] = 1.0 / at + (t > 0 ? hb[(t - 1) * gp::kMaxCols + c] / ha[(t - 1) * gp::kMaxCols + c] : 0.0);
      e[t] = t + 1 < m ? sqrt(hb[t * gp::kMaxCols + c]) / at : 0.0;
    }
    bool ok = m > 0 && tridiag_ql(d, e, z, m);
    double g = 0.0;
    for (int t = 0; t < m && ok; ++t) {
      if (!(d[t] > 0.0)) ok = false;
      else g += z[t] * z[t] * log(d[t]);
    }
    gam[2 * l] = g * (double)n_act;
    gam[2 * l + 1] = ok ? 0.0 : 1.0;
    __threadfence();
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) last = atomicInc(&s->ticket4, gridDim.x - 1) == gridDim.x - 1;
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double mean = 0.0;
    int nbad = 0;
    for (int q = 0; q < nv; ++q) {
      mean += __ldcg(gam + 2 * q);
      nbad += __ldcg(gam + 2 * q + 1) != 0.0;
    }
    mean /= nv;
    double var = 0.0;
    for (int q = 0; q < nv; ++q) {
      const double dq = __ldcg(gam + 2 * q) - mean;
      var += dq * dq;
    }
    var = nv > 1 ? var / (nv - 1) : 0.0;
    s->slq_mean = mean;
    s->slq_var = var;
    s->status = nbad ? GP_ERR_NOT_SPD : GP_OK;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_alpha_active(int64_t n, const uint32_t* __restrict__ perm,
                                                           const double* __restrict__ dinv64,
                                                           const T* __restrict__ X, int64_t ld,
                                                           double* __restrict__ out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    out[perm[p]] = dinv64[p] * (double)X[p * ld];
}

__global__ void __launch_bounds__(kThreads) k_alpha_inactive(int64_t n, const uint32_t* __restrict__ mask0,
                                                             const double* __restrict__ y, double inv_s2,
                                                             double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (mask0[i] == 0u) out[i] = y[i] * inv_s2;
}

unsigned grid_for(int64_t items, int per_block, int max_blocks) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (unsigned)g;
}

int read_state(gp_ctx* c, gp::CgState* host) {
  GP_CHECK(gp::ensure_pinned(c, sizeof(gp::CgState)));
  GP_CUDA(cudaMemcpyAsync(c->pinned, c->cg.p, sizeof(gp::CgState), cudaMemcpyDeviceToHost, c->stream));
  GP_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(host, c->pinned, sizeof(gp::CgState));
  return GP_OK;
}

}  // namespace

namespace gp {

namespace {

// What the iterations of one FP32 CG run launch, fixed by its preparation.
struct CgLoop {
  SpmmPlan plan;
  bool pc = false;
  int kq = 0;
  unsigned g_pc = 0, g_upd = 0, g_upd_r = 0;
  size_t pc_smem = 0;
  UpdPcFn upd_pc = nullptr;
};

// Everything of a run before its iterations (c->n_act > 0): buffers, the
// starting state and residual (warm start, caller block, or [yhat, probes]),
// the preconditioned start, and the launch shapes of the iterations, with the
// SpMM form chosen under spmm_flags.
int cg_prepare(gp_ctx* c, int k, int kp, const double* y, int nv, uint64_t seed, int m_hist, int max_iter,
               double rtol, bool use_pc, bool warm, const float* rhs, int spmm_flags, CgLoop* L) {
  const int64_t n = c->n_act;
  if (!spmm_available(GP_SPMM_CPASYNC, kp)) return GP_ERR_UNSUPPORTED;
  GP_CHECK(ensure(c, c->X, (size_t)n * kp * sizeof(float)));
  GP_CHECK(ensure(c, c->R, (size_t)n * kp * sizeof(float)));
  GP_CHECK(ensure(c, c->P, (size_t)n * kp * sizeof(float)));
  GP_CHECK(ensure(c, c->Q, (size_t)n * kp * sizeof(float)));
  GP_CHECK(ensure(c, c->zbits, (size_t)n * 2 * sizeof(uint32_t)));
  const int maxb = c->num_sms * 4;
  GP_CHECK(ensure(c, c->part_a, (size_t)maxb * 4 * kMaxCols * sizeof(double)));
  GP_CHECK(ensure(c, c->part_b, (size_t)c->num_sms * 8 * kMaxCols * sizeof(double)));
  GP_CHECK(ensure(c, c->hist_alpha, (size_t)kMaxLanczos * kMaxCols * sizeof(double)));
  GP_CHECK(ensure(c, c->hist_beta, (size_t)kMaxLanczos * kMaxCols * sizeof(double)));
  CgState* st = (CgState*)c->cg.p;
  const Group none{nullptr, nullptr};
  // the warm start keeps rr0 = |B|^2 and relies on the preconditioned start
  // to set rho_0 from the new residual
  if (warm && !(use_pc && c->pc_block > 0)) return GP_ERR_INVALID_ARG;
  if (warm) {
    // continue from the iterate X of the previous run on the same block:
    // Q = Khat X (the product runs while the state says iteration 0 of an
    // unfinished run), then the init forms R = B - Q
    GP_CUDA(cudaMemsetAsync(&st->iter, 0, sizeof(st->iter), c->stream));
    GP_CUDA(cudaMemsetAsync(&st->fin[0], 0, sizeof(st->fin), c->stream));
    SpmmPlan wp;
    GP_CHECK(spmm_plan(c, kp, GP_SPMM_CPASYNC, &wp));
    spmm_launch_io(wp, c->stream, c, st, (const float*)c->X.p, (float*)c->Q.p);
    GP_LAUNCH_CHECK();
    c->launches += 1;
  }
  if (rhs) {
    // a caller-given right-hand-side block: no probes, no Lanczos record
    if (warm || m_hist != 0) return GP_ERR_INVALID_ARG;
    const int kqr = kp / 4;
    const unsigned gr = grid_for(n, kUpdRThreads / kqr, c->num_sms);
    k_rhs_init_f32<<<gr, kUpdRThreads, 0, c->stream>>>(n, kqr, (const float4*)rhs, (float4*)c->X.p,
                                                       (float4*)c->R.p, (float4*)c->P.p, (double*)c->part_a.p);
    k_rhs_state<<<1, kRedThreads, 0, c->stream>>>((const double*)c->part_a.p, (int)gr, k, kp, st, rtol * rtol,
                                                  max_iter);
    GP_LAUNCH_CHECK();
    c->launches += 2;
  } else {
    unsigned gb = grid_for(n, kThreads, maxb);
    k_init_f32<<<gb, kThreads, 0, c->stream>>>(n, k, kp, y, (const uint32_t*)c->vals.p, (const double*)c->dinv64.p,
                                               seed, nv, (float*)c->X.p, (float*)c->R.p, (float*)c->P.p,
                                               warm ? (const float*)c->Q.p : nullptr, (uint32_t*)c->zbits.p,
                                               (double*)c->part_a.p, st, rtol * rtol, max_iter);
    GP_LAUNCH_CHECK();
    c->launches += 1;
  }
  // block-Jacobi preconditioned CG: Z = M^-1 R, beta from r^T z, stop on |r|
  L->pc = use_pc && c->pc_block > 0;
  L->kq = kp / 4;
  const int kq = L->kq;
  L->g_pc = 0;
  L->pc_smem = 0;
  L->upd_pc = nullptr;
  if (L->pc) {
    L->pc_smem = pc_smem_bytes(kq, c->pc_block);
    int smem_max = 0;
    GP_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    if (L->pc_smem > (size_t)smem_max) return GP_ERR_UNSUPPORTED;
    UpdPcFn upd_pc_init = upd_pc_fn<true>(c->pc_block);
    L->upd_pc = upd_pc_fn<false>(c->pc_block);
    if (!upd_pc_init || !L->upd_pc) return GP_ERR_UNSUPPORTED;
    GP_CUDA(cudaFuncSetAttribute(upd_pc_init, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L->pc_smem));
    GP_CUDA(cudaFuncSetAttribute(L->upd_pc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L->pc_smem));
    // two blocks per SM, two tiles each in flight: enough bytes in flight for
    // HBM without many partial rows for the one-block reduction
    L->g_pc = grid_for(n, pc_tile(c->pc_block), c->num_sms * 2);
    GP_CHECK(ensure(c, c->Z, (size_t)n * kp * sizeof(float)));
    GP_CHECK(ensure(c, c->part_b, (size_t)L->g_pc * 2 * kp * sizeof(double)));
    upd_pc_init<<<L->g_pc, kPcLanes * kq, L->pc_smem, c->stream>>>(n, kq, nullptr, (float4*)c->R.p,
                                                                     (float4*)c->P.p, (const float*)c->pc_Minv.p,
                                                                     (double*)c->part_b.p, st, none);
    k_pc_state<<<1, kRedThreads, 0, c->stream>>>((const double*)c->part_b.p, (int)L->g_pc, k, kp, st);
    GP_LAUNCH_CHECK();
    c->launches += 2;
  }
  // the SpMM form: forced by the flags, else the autotuner's for this shape
  GP_CHECK(spmm_select(c, kp, spmm_flags, st, &L->plan, k, m_hist));
  c->spmm_variant = L->plan.variant;
  L->g_upd = grid_for(n, kUpdThreads / kq, c->num_sms * 8);
  L->g_upd_r = grid_for(n, kUpdRThreads / kq, c->num_sms);
  return GP_OK;
}

// The outcome of a run from its final state: iterations, the largest relative
// residual over the k columns, and the run's status.
int cg_finish(gp_ctx* c, int k, int* iters_out, double* max_rel) {
  CgState hs;
  GP_CHECK(read_state(c, &hs));
  *iters_out = hs.iter;
  double mr = 0.0;
  bool all_done = true;
  const int par = hs.iter & 1;
  for (int q = 0; q < k; ++q) {
    if (hs.rr0[q] > 0) mr = fmax(mr, sqrt(hs.crr[par][q] / hs.rr0[q]));
    all_done = all_done && hs.donep[par][q];
  }
  *max_rel = mr;
  c->bad_col = hs.bad_col;
  c->bad_iter = hs.iter;
  if (hs.status != GP_OK) return hs.status;
  if (!all_done) return GP_ERR_NOT_CONVERGED;
  return GP_OK;
}

}  // namespace

int cg_run(gp_ctx* c, int k, int kp, const double* y, int nv, uint64_t seed, int m_hist, int max_iter, double rtol,
           int check_every, int* iters_out, double* max_rel, bool use_pc, bool warm, const float* rhs) {
  const int64_t n = c->n_act;
  *iters_out = 0;
  *max_rel = 0.0;
  if (n == 0) return GP_OK;
  CgLoop L;
  GP_CHECK(cg_prepare(c, k, kp, y, nv, seed, m_hist, max_iter, rtol, use_pc, warm, rhs, c->flags, &L));
  CgState* st = (CgState*)c->cg.p;
  const Group none{nullptr, nullptr};
  const int64_t nblk = c->nblk;
  const SpmmPlan& plan = L.plan;
  const bool pc = L.pc;
  const int kq = L.kq;
  const unsigned g_spmm = plan.grid, g_pc = L.g_pc, g_upd = L.g_upd, g_upd_r = L.g_upd_r;
  const size_t pc_smem = L.pc_smem;
  if (check_every <= 0) check_every = 16;
  if (check_every > 64) check_every = 64;
  const bool timed = (c->flags & GP_FLAG_TIME_KERNELS) != 0;
  if (timed) GP_CHECK(kernel_events(c));
  // one CG iteration: the kernels read the iteration index from the device
  // state, so the same launches serve every iteration (and a graph of them)
  // (events recorded during capture become external event-record nodes,
  // which time like ordinary records)
  auto launch_iteration = [&](cudaStream_t sm, cudaEvent_t ev0, cudaEvent_t ev1) {
    const unsigned evf = sm == c->cap_stream ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (ev0) cudaEventRecordWithFlags(ev0, sm, evf);
    spmm_launch(plan, sm, c, st);
    if (ev1) cudaEventRecordWithFlags(ev1, sm, evf);
    if (!plan.fused_alpha)
      k_cg_alpha_cols<<<kp, kColThreads, 0, sm>>>((const double*)c->part_a.p, (int)g_spmm, k, kp, st,
                                                  (double*)c->hist_alpha.p, m_hist, none);
    if (pc) {
      L.upd_pc<<<g_pc, kPcLanes * kq, pc_smem, sm>>>(n, kq, (const float4*)c->Q.p, (float4*)c->R.p,
                                                     (float4*)c->Z.p, (const float*)c->pc_Minv.p,
                                                     (double*)c->part_b.p, st, none);
      k_cg_beta_cols<<<kp, kColThreads, 0, sm>>>((const double*)c->part_b.p, (int)g_pc, k, kp, 1, st,
                                                 (double*)c->hist_beta.p, m_hist, none);
    } else {
      k_upd_r_f32<<<g_upd_r, kUpdRThreads, 0, sm>>>(n, kq, (const float4*)c->Q.p, (float4*)c->R.p,
                                                    (double*)c->part_b.p, st, none);
      k_cg_beta_cols<<<kp, kColThreads, 0, sm>>>((const double*)c->part_b.p, (int)g_upd_r, k, kp, 0, st,
                                                 (double*)c->hist_beta.p, m_hist, none);
    }
    k_upd_xp_f32<<<g_upd, kUpdThreads, 0, sm>>>(n, kq, (float4*)c->X.p, (const float4*)(pc ? c->Z.p : c->R.p),
                                                (float4*)c->P.p, st, none);
  };
  // graph of check_every iterations, rebuilt only when an argument changes
  // (with GP_FLAG_TIME_KERNELS the graph also records the SpMM events)
  cudaGraphExec_t exec = nullptr;
  {
    const uint64_t key[48] = {(uint64_t)n, (uint64_t)nblk, (uint64_t)k, (uint64_t)kp, (uint64_t)pc,
                              (uint64_t)c->pc_block, (uint64_t)g_spmm, (uint64_t)g_pc, (uint64_t)g_upd,
                              (uint64_t)g_upd_r, (uint64_t)m_hist, (uint64_t)check_every, (uint64_t)plan.smem,
                              (uint64_t)pc_smem, (uint64_t)(uintptr_t)plan.fn, (uint64_t)(uintptr_t)c->brp.p,
                              (uint64_t)(uintptr_t)c->bcol.p, (uint64_t)(uintptr_t)c->bval.p,
                              (uint64_t)(uintptr_t)c->P.p, (uint64_t)(uintptr_t)c->Q.p, (uint64_t)(uintptr_t)c->R.p,
                              (uint64_t)(uintptr_t)c->X.p, (uint64_t)(uintptr_t)c->Z.p,
                              (uint64_t)(uintptr_t)c->part_a.p, (uint64_t)(uintptr_t)c->part_b.p,
                              (uint64_t)(uintptr_t)c->hist_alpha.p, (uint64_t)(uintptr_t)c->hist_beta.p,
                              (uint64_t)(uintptr_t)st, (uint64_t)(uintptr_t)c->pc_Minv.p, (uint64_t)timed,
                              (uint64_t)(uintptr_t)(timed ? c->kev[0] : nullptr), (uint64_t)plan.variant,
                              (uint64_t)plan.stages, (uint64_t)plan.grid, (uint64_t)c->w_ntiles,
                              (uint64_t)c->w_nrun, (uint64_t)(uintptr_t)c->w_tseg.p,
                              (uint64_t)(uintptr_t)c->w_segd.p, (uint64_t)(uintptr_t)c->w_runs.p,
                              (uint64_t)(uintptr_t)c->w_rec.p, 0};
    gp_ctx::CgGraph& gr = c->cg_graph[pc ? 1 : 0];
    if (gr.exec && memcmp(gr.key, key, sizeof(key)) != 0) {
      GP_CUDA(cudaGraphExecDestroy(gr.exec));
      gr.exec = nullptr;
    }
    if (!gr.exec) {
      if (!c->cap_stream) GP_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
      cudaGraph_t graph = nullptr;
      GP_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      for (int t = 0; t < check_every; ++t)
        launch_iteration(c->cap_stream, timed ? c->kev[2 * t] : nullptr, timed ? c->kev[2 * t + 1] : nullptr);
      GP_CUDA(cudaStreamEndCapture(c->cap_stream, &graph));
      const cudaError_t ie = cudaGraphInstantiate(&gr.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) {
        gr.exec = nullptr;
        return GP_ERR_CUDA;
      }
      memcpy(gr.key, key, sizeof(key));
    }
    exec = gr.exec;
  }
  CgState hs;
  int iter_before = 0;
  for (int it0 = 0; it0 < max_iter; it0 += check_every) {
    if (exec) {
      GP_CUDA(cudaGraphLaunch(exec, c->stream));
    } else {
      for (int t = 0; t < check_every; ++t) launch_iteration(c->stream, c->kev[2 * t], c->kev[2 * t + 1]);
      GP_LAUNCH_CHECK();
    }
    c->launches += (plan.fused_alpha ? 4 : 5) * check_every;
    GP_CHECK(read_state(c, &hs));
    if (timed) {
      // launches after convergence return at once: time only the ones that worked
      const int worked = hs.iter - iter_before;
      for (int t = 0; t < worked && t < check_every; ++t) c->t_spmm += event_ms(c->kev[2 * t], c->kev[2 * t + 1]);
      c->n_spmm += worked < check_every ? worked : check_every;
    }
    iter_before = hs.iter;
    if (hs.finished) break;
  }
  return cg_finish(c, k, iters_out, max_rel);
}

namespace {

// finished flag of every instance of a group (1 for those not in it)
__global__ void k_group_done(const GInst* __restrict__ inst, int nc, int* __restrict__ out) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) out[i] = inst[i].st ? inst[i].st->finished : 1;
}

// CTA maps of a grouped launch over the live instances: for each kind, the
// instance's own grid in order (entry (i << kGroupShift) | b for CTA b of
// instance i).  kColMap: the per-column kernels (kp CTAs per instance).
constexpr int kColMap = 4;
void group_maps(const std::vector<GInst>& inst, const std::vector<int>& live, int kp, std::vector<uint32_t>& maps,
                size_t off[6]) {
  maps.clear();
  for (int kind = 0; kind < 5; ++kind) {
    off[kind] = maps.size();
    for (int i : live) {
      const int g = kind == kColMap ? kp : inst[i].grid[kind];
      for (int b = 0; b < g; ++b) maps.push_back(((uint32_t)i << kGroupShift) | (uint32_t)b);
    }
  }
  off[5] = maps.size();
}

}  // namespace

int cg_run_group(gp_ctx* owner, gp_ctx* const* cs, int nc, int k, int kp, const double* const* ys, int nv,
                 uint64_t seed, int m_hist, int max_iter, double rtol, int check_every, bool use_pc, bool warm,
                 int* iters, double* max_rel, int* status) {
  if (nc < 0 || nc > kMaxGroup) return GP_ERR_INVALID_ARG;
  if (nc == 0) return GP_OK;
  if (check_every <= 0) check_every = 16;
  if (check_every > 64) check_every = 64;
  cudaStream_t s = owner->stream;
  std::vector<CgLoop> L(nc);
  std::vector<GInst> inst(nc);
  std::vector<int> live;
  std::vector<cudaEvent_t> ready(nc, nullptr);
  int first = -1;
  int result = GP_OK;
  for (int i = 0; i < nc && result == GP_OK; ++i) {
    gp_ctx* c = cs[i];
    iters[i] = 0;
    max_rel[i] = 0.0;
    status[i] = GP_OK;
    GInst& I = inst[i];
    memset(&I, 0, sizeof(I));
    if (c->n_act == 0) continue;
    // the same preparation as a run on its own, with the cp.async product
    status[i] = cg_prepare(c, k, kp, ys[i], nv, seed, m_hist, max_iter, rtol, use_pc, warm, nullptr,
                           GP_FLAG_SPMM_CPASYNC_WIDE, &L[i]);
    if (status[i] != GP_OK) continue;
    if (first < 0) first = i;
    // every instance of one grouped launch runs the same kernel
    const CgLoop& L0 = L[first];
    if (L[i].plan.fn != L0.plan.fn || L[i].plan.smem != L0.plan.smem || L[i].pc != L0.pc ||
        L[i].upd_pc != L0.upd_pc || L[i].pc_smem != L0.pc_smem) {
      result = GP_ERR_UNSUPPORTED;
      break;
    }
    I.n = c->n_act;
    I.nblk = c->nblk;
    I.brp = (const int64_t*)c->brp.p;
    I.bcol = (const int32_t*)c->bcol.p;
    I.bval = (const float4*)c->bval.p;
    I.X = (float4*)c->X.p;
    I.R = (float4*)c->R.p;
    I.P = (float4*)c->P.p;
    I.Q = (float4*)c->Q.p;
    I.Z = L[i].pc ? (float4*)c->Z.p : nullptr;
    I.D = L[i].pc ? I.Z : I.R;
    I.Minv = (const float*)c->pc_Minv.p;
    I.part_a = (double*)c->part_a.p;
    I.part_b = (double*)c->part_b.p;
    I.hist_alpha = (double*)c->hist_alpha.p;
    I.hist_beta = (double*)c->hist_beta.p;
    I.st = (CgState*)c->cg.p;
    I.grid[kGSpmm] = (int)L[i].plan.grid;
    I.grid[kGPc] = (int)L[i].g_pc;
    I.grid[kGUpd] = (int)L[i].g_upd;
    I.grid[kGUpdR] = (int)L[i].g_upd_r;
    live.push_back(i);
    // the group's stream starts after the instance's preparation
    cudaError_t ce = cudaEventCreateWithFlags(&ready[i], cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventRecord(ready[i], c->stream);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, ready[i], 0);
    if (ce != cudaSuccess) {
      result = cuda_status(ce);
      break;
    }
  }
  // the iterations; a failure inside still reaches the ordering below, so no
  // instance's buffers are reused while a grouped launch may read them
  auto iterate = [&]() -> int {
    const CgLoop& L0 = L[first];
    const int kq = L0.kq;
    const bool pc = L0.pc;
    // instance table (uploaded once) and the finished flags after it
    const size_t tab_bytes = (size_t)nc * sizeof(GInst);
    GP_CHECK(ensure(owner, owner->grp_inst, tab_bytes + (size_t)nc * sizeof(int)));
    GInst* dinst = (GInst*)owner->grp_inst.p;
    int* ddone = (int*)((char*)owner->grp_inst.p + tab_bytes);
    GP_CUDA(cudaMemcpyAsync(dinst, inst.data(), tab_bytes, cudaMemcpyHostToDevice, s));
    std::vector<uint32_t> maps;
    size_t off[6];
    std::vector<int> done(nc);
    bool rebuild = true;
    const int max_checks = max_iter / check_every + 2;
    for (int chk = 0; chk < max_checks && !live.empty(); ++chk) {
      if (rebuild) {
        // the CTA maps of the instances still running (the launches of the
        // last check interval have completed: their flags were read)
        group_maps(inst, live, kp, maps, off);
        // (the first build is the largest: buffers never grow while a copy
        // from or to them is queued)
        GP_CHECK(ensure(owner, owner->grp_map, maps.size() * sizeof(uint32_t)));
        GP_CHECK(ensure_pinned(owner, std::max(maps.size() * sizeof(uint32_t), (size_t)nc * sizeof(int))));
        memcpy(owner->pinned, maps.data(), maps.size() * sizeof(uint32_t));
        GP_CUDA(cudaMemcpyAsync(owner->grp_map.p, owner->pinned, maps.size() * sizeof(uint32_t),
                                cudaMemcpyHostToDevice, s));
        rebuild = false;
      }
      const uint32_t* dmap = (const uint32_t*)owner->grp_map.p;
      const Group gs{dinst, dmap + off[kGSpmm]}, gc{dinst, dmap + off[kColMap]}, gpc{dinst, dmap + off[kGPc]},
          gu{dinst, dmap + off[kGUpd]}, gr{dinst, dmap + off[kGUpdR]};
      const unsigned n_spmm = (unsigned)(off[kGSpmm + 1] - off[kGSpmm]);
      const unsigned n_pc = (unsigned)(off[kGPc + 1] - off[kGPc]);
      const unsigned n_upd = (unsigned)(off[kGUpd + 1] - off[kGUpd]);
      const unsigned n_updr = (unsigned)(off[kGUpdR + 1] - off[kGUpdR]);
      const unsigned n_col = (unsigned)(off[kColMap + 1] - off[kColMap]);
      for (int t = 0; t < check_every; ++t) {
        // one iteration of every live instance: the launches of cg_run, each
        // CTA taking its instance's arguments from the table
        spmm_launch_group(L0.plan, s, n_spmm, gs);
        k_cg_alpha_cols<<<n_col, kColThreads, 0, s>>>(nullptr, 0, k, kp, nullptr, nullptr, m_hist, gc);
        if (pc) {
          L0.upd_pc<<<n_pc, kPcLanes * kq, L0.pc_smem, s>>>(0, kq, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                            nullptr, gpc);
          k_cg_beta_cols<<<n_col, kColThreads, 0, s>>>(nullptr, 0, k, kp, 1, nullptr, nullptr, m_hist, gc);
        } else {
          k_upd_r_f32<<<n_updr, kUpdRThreads, 0, s>>>(0, kq, nullptr, nullptr, nullptr, nullptr, gr);
          k_cg_beta_cols<<<n_col, kColThreads, 0, s>>>(nullptr, 0, k, kp, 0, nullptr, nullptr, m_hist, gc);
        }
        k_upd_xp_f32<<<n_upd, kUpdThreads, 0, s>>>(0, kq, nullptr, nullptr, nullptr, nullptr, gu);
      }
      GP_LAUNCH_CHECK();
      k_group_done<<<1, 256, 0, s>>>(dinst, nc, ddone);
      GP_LAUNCH_CHECK();
      owner->launches += 5 * check_every + 1;
      GP_CUDA(cudaMemcpyAsync(owner->pinned, ddone, (size_t)nc * sizeof(int), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaStreamSynchronize(s));
      memcpy(done.data(), owner->pinned, (size_t)nc * sizeof(int));
      std::vector<int> still;
      for (int i : live)
        if (!done[i]) still.push_back(i);
      rebuild = still.size() != live.size();
      live.swap(still);
    }
    return GP_OK;
  };
  if (result == GP_OK && !live.empty()) result = iterate();
  // every instance's stream continues after the group's launches
  cudaEvent_t after = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&after, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(after, s);
  if (e != cudaSuccess) {
    // no event to order by: wait for the group's stream instead
    cudaStreamSynchronize(s);
    if (result == GP_OK) result = cuda_status(e);
  }
  for (int i = 0; i < nc; ++i) {
    if (ready[i]) cudaEventDestroy(ready[i]);
    if (cs[i]->n_act == 0 || status[i] != GP_OK) continue;
    if (e == cudaSuccess) {
      const cudaError_t w = cudaStreamWaitEvent(cs[i]->stream, after, 0);
      if (w != cudaSuccess && result == GP_OK) result = cuda_status(w);
    }
    if (result == GP_OK) status[i] = cg_finish(cs[i], k, &iters[i], &max_rel[i]);
  }
  if (after) cudaEventDestroy(after);
  return result;
}

int cg_run_fp64(gp_ctx* c, int k, const double* y, int nv, uint64_t seed, int m_hist, int max_iter, double rtol,
                int check_every, int* iters_out, double* max_rel, const double* rhs) {
  const int64_t n = c->n_act;
  *iters_out = 0;
  *max_rel = 0.0;
  if (n == 0) return GP_OK;
  GP_CHECK(ensure(c, c->X, (size_t)n * k * sizeof(double)));
  GP_CHECK(ensure(c, c->R, (size_t)n * sizeof(double)));
  GP_CHECK(ensure(c, c->P, (size_t)n * sizeof(double)));
  GP_CHECK(ensure(c, c->Q, (size_t)n * sizeof(double)));
  GP_CHECK(ensure(c, c->zbits, (size_t)n * 2 * sizeof(uint32_t)));
  const int maxb = c->num_sms * 4;
  GP_CHECK(ensure(c, c->part_a, (size_t)maxb * 4 * kMaxCols * sizeof(double)));
  GP_CHECK(ensure(c, c->part_b, (size_t)maxb * 4 * kMaxCols * sizeof(double)));
  GP_CHECK(ensure(c, c->hist_alpha, (size_t)kMaxLanczos * kMaxCols * sizeof(double)));
  GP_CHECK(ensure(c, c->hist_beta, (size_t)kMaxLanczos * kMaxCols * sizeof(double)));
  CgState* st = (CgState*)c->cg.p;
  if (check_every <= 0) check_every = 16;
  if (check_every > 64) check_every = 64;
  const unsigned gb = grid_for(n, kThreads, maxb);
  const unsigned gw = grid_for(n, kWarps, c->num_sms * 4);
  int status = GP_OK;
  double mr = 0.0;
  int itmax = 0;
  for (int col = 0; col < k; ++col) {
    double* X = (double*)c->X.p + (int64_t)col * n;
    k_init_f64<<<gb, kThreads, 0, c->stream>>>(n, col, nv, y, (const uint32_t*)c->vals.p,
                                               (const double*)c->dinv64.p, rhs, seed, X, (double*)c->R.p,
                                               (double*)c->P.p, (uint32_t*)c->zbits.p, (double*)c->part_a.p, st,
                                               rtol * rtol, max_iter);
    GP_LAUNCH_CHECK();
    c->launches += 1;
    CgState hs;
    for (int it = 0; it < max_iter; it += check_every) {
      for (int t = 0; t < check_every; ++t) {
        k_spmv_f64<<<gw, kThreads, 0, c->stream>>>(n, (const int64_t*)c->row_ptr.p, (const int32_t*)c->col.p,
                                                   (const double*)c->val.p, (const double*)c->P.p, (double*)c->Q.p,
                                                   (double*)c->part_a.p, st, col, (double*)c->hist_alpha.p, m_hist);
        k_upd_r_f64<<<gb, kThreads, 0, c->stream>>>(n, (const double*)c->Q.p, (double*)c->R.p,
                                                    (double*)c->part_b.p, st, col, (double*)c->hist_beta.p, m_hist);
        k_upd_xp_f64<<<gb, kThreads, 0, c->stream>>>(n, X, (const double*)c->R.p, (double*)c->P.p, st);
      }
      GP_LAUNCH_CHECK();
      c->launches += 3 * check_every;
      GP_CHECK(read_state(c, &hs));
      if (hs.finished) break;
    }
    GP_CHECK(read_state(c, &hs));
    itmax = hs.iter > itmax ? hs.iter : itmax;
    if (hs.rr0[0] > 0) mr = fmax(mr, sqrt(hs.rr[0] / hs.rr0[0]));
    if (hs.status != GP_OK && status == GP_OK) status = hs.status;
    if (!hs.done[0] && status == GP_OK) status = GP_ERR_NOT_CONVERGED;
  }
  *iters_out = itmax;
  *max_rel = mr;
  return status;
}

int inactive_terms(gp_ctx* c, const double* y) {
  AsmScalars* s = (AsmScalars*)c->asm_s.p;
  const int maxb = c->num_sms * 4;
  GP_CHECK(ensure(c, c->part_c, (size_t)maxb * 2 * sizeof(double)));
  if (c->n == 0) {
    GP_CUDA(cudaMemsetAsync(&s->inact_y2, 0, sizeof(double), c->stream));
    GP_CUDA(cudaMemsetAsync(&s->n_inactive, 0, sizeof(long long), c->stream));
    return GP_OK;
  }
  k_inactive<<<grid_for(c->n, kThreads, maxb), kThreads, 0, c->stream>>>(c->n, y, (const uint32_t*)c->mask0.p,
                                                                         (double*)c->part_c.p, s);
  GP_LAUNCH_CHECK();
  c->launches += 1;
  return GP_OK;
}

int quad_form(gp_ctx* c, const double* y, int kp) {
  AsmScalars* s = (AsmScalars*)c->asm_s.p;
  if (c->n_act == 0) {
    GP_CUDA(cudaMemsetAsync(&s->quad_form, 0, sizeof(double), c->stream));
    return GP_OK;
  }
  const int maxb = c->num_sms * 4;
  GP_CHECK(ensure(c, c->part_c, (size_t)maxb * 2 * sizeof(double)));
  const unsigned gb = grid_for(c->n_act, kThreads, maxb);
  if (c->precision == GP_FP64)
    k_quad<double><<<gb, kThreads, 0, c->stream>>>(c->n_act, y, (const uint32_t*)c->vals.p,
                                                   (const double*)c->dinv64.p, (const double*)c->X.p, 1,
                                                   (double*)c->part_c.p, s);
  else
    k_quad<float><<<gb, kThreads, 0, c->stream>>>(c->n_act, y, (const uint32_t*)c->vals.p,
                                                  (const double*)c->dinv64.p, (const float*)c->X.p, kp,
                                                  (double*)c->part_c.p, s);
  GP_LAUNCH_CHECK();
  c->launches += 1;
  return GP_OK;
}

int slq(gp_ctx* c, int nv, int kcols, bool overlap) {
  (void)kcols;
  AsmScalars* s = (AsmScalars*)c->asm_s.p;
  if (c->n_act == 0) {
    GP_CUDA(cudaMemsetAsync(&s->slq_mean, 0, 2 * sizeof(double), c->stream));
    return GP_OK;
  }
  GP_CHECK(ensure(c, c->slq_g, (size_t)2 * kMaxProbes * sizeof(double)));
  const int* steps = ((const CgState*)c->cg.p)->steps;
  cudaStream_t sm = c->stream;
  if (overlap) {
    // the eigen-solves are serial FP64 work on 32 SMs: run them on the side
    // stream while the next solve runs; they read the Lanczos coefficients
    // (not written again before the join) and a copy of the step counts
    if (!c->aux_stream) {
      GP_CUDA(cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
      GP_CUDA(cudaEventCreateWithFlags(&c->aux_ev[0], cudaEventDisableTiming));
      GP_CUDA(cudaEventCreateWithFlags(&c->aux_ev[1], cudaEventDisableTiming));
    }
    GP_CHECK(ensure(c, c->slq_steps, (size_t)kMaxCols * sizeof(int)));
    GP_CUDA(cudaMemcpyAsync(c->slq_steps.p, steps, (size_t)kMaxCols * sizeof(int), cudaMemcpyDeviceToDevice,
                            c->stream));
    GP_CUDA(cudaEventRecord(c->aux_ev[0], c->stream));
    GP_CUDA(cudaStreamWaitEvent(c->aux_stream, c->aux_ev[0], 0));
    steps = (const int*)c->slq_steps.p;
    sm = c->aux_stream;
  }
  k_slq<<<nv, 32, 0, sm>>>(nv, c->n_act, (const double*)c->hist_alpha.p, (const double*)c->hist_beta.p, steps,
                           (double*)c->slq_g.p, s);
  GP_LAUNCH_CHECK();
  c->launches += 1;
  if (overlap) {
    GP_CUDA(cudaEventRecord(c->aux_ev[1], c->aux_stream));
    c->slq_pending = true;
  }
  return GP_OK;
}

int slq_join(gp_ctx* c) {
  if (!c->slq_pending) return GP_OK;
  c->slq_pending = false;
  GP_CUDA(cudaStreamWaitEvent(c->stream, c->aux_ev[1], 0));
  return GP_OK;
}

int alpha_out(gp_ctx* c, const double* y, double* out, int kp) {
  const int maxb = c->num_sms * 4;
  if (c->n > 0)
    k_alpha_inactive<<<grid_for(c->n, kThreads, maxb), kThreads, 0, c->stream>>>(
        c->n, (const uint32_t*)c->mask0.p, y, 1.0 / c->sigma2, out);
  if (c->n_act > 0) {
    const unsigned gb = grid_for(c->n_act, kThreads, maxb);
    if (c->precision == GP_FP64)
      k_alpha_active<double><<<gb, kThreads, 0, c->stream>>>(c->n_act, (const uint32_t*)c->vals.p,
                                                             (const double*)c->dinv64.p, (const double*)c->X.p, 1,
                                                             out);
    else
      k_alpha_active<float><<<gb, kThreads, 0, c->stream>>>(c->n_act, (const uint32_t*)c->vals.p,
                                                            (const double*)c->dinv64.p, (const float*)c->X.p, kp,
                                                            out);
  }
  GP_LAUNCH_CHECK();
  c->launches += (c->n > 0) + (c->n_act > 0);
  return GP_OK;
}

}  // namespace gp
