// Sparse assembly of K (Sec. 2.2, Eq. eq:bump_kernel with Eq. eq:bump and
// Eq. eq:kstat) on one GPU:
//   bbox -> bump table (F, support mask) -> active compaction -> Morton keys
//   -> LSD radix sort -> cell table -> per-row pair count -> scan -> fill.
// The stored matrix is the Jacobi-scaled active block
//   Khat = D^-1/2 K_act D^-1/2,  D = diag(K_act) = A C sum_m F_m^2 + sigma_n^2,
// in CSR with rows and columns in Morton order and ascending columns.
#include <math.h>

#include <algorithm>
#include <climits>
#include <utility>
#include <vector>

#include "gp_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ bbox
__global__ void __launch_bounds__(kThreads) k_bbox(const double* __restrict__ x, int64_t n, int dim,
                                                   double* __restrict__ part, gp::AsmScalars* s) {
  double lo[gp::kMaxDim], hi[gp::kMaxDim];
  for (int k = 0; k < gp::kMaxDim; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < dim; ++k) {
      double v = x[i * dim + k];
      lo[k] = fmin(lo[k], v);
      hi[k] = fmax(hi[k], v);
    }
  }
  __shared__ double sh[kThreads];
  __shared__ bool last;
  for (int k = 0; k < dim; ++k) {
    for (int side = 0; side < 2; ++side) {
      sh[threadIdx.x] = side ? hi[k] : lo[k];
      __syncthreads();
      for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
          double a = sh[threadIdx.x], b = sh[threadIdx.x + o];
          sh[threadIdx.x] = side ? fmax(a, b) : fmin(a, b);
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) part[(blockIdx.x * gp::kMaxDim + k) * 2 + side] = sh[0];
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicInc(&s->ticket0, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  // the last block: every thread folds a strided share of the partials, then
  // a tree per axis and side
  __threadfence();
  for (int k = 0; k < dim; ++k) {
    for (int side = 0; side < 2; ++side) {
      double v = side ? -INFINITY : INFINITY;
      for (unsigned g = threadIdx.x; g < gridDim.x; g += blockDim.x) {
        const double t = __ldcg(part + (g * gp::kMaxDim + k) * 2 + side);
        v = side ? fmax(v, t) : fmin(v, t);
      }
      sh[threadIdx.x] = v;
      __syncthreads();
      for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
          const double a = sh[threadIdx.x], b = sh[threadIdx.x + o];
          sh[threadIdx.x] = side ? fmax(a, b) : fmin(a, b);
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        if (side) s->bbox_hi[k] = sh[0];
        else s->bbox_lo[k] = sh[0];
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ bump table
// F0[i, m] = f_m(x_i) (Eq. eq:bump, support |x - c| < r), mask0[i] bit m set
// iff x_i lies inside some bump of f_m; flag[i] = (mask0[i] != 0).
// An FP32 pre-filter (coordinates relative to the bounding box) rejects bumps
// far from the point; every accepted bump is re-tested and evaluated in FP64
// with the same operation order as the plain definition.
// GB300's FP64 pipe takes about 16 cycles per warp instruction, and a branch
// taken by one lane costs the whole warp, so the accepted (point, bump) pairs
// of a warp are queued in shared memory and evaluated 32 at a time with all
// lanes busy (about one FP64 pass per warp instead of one per bump that any
// lane accepts).  Each lane then adds its own results in bump order, so the
// compensated sums are those of a plain loop over the bumps.
constexpr int kBtQueue = 96;  // queued pairs per warp (flushed before it can overflow)

__global__ void __launch_bounds__(kThreads) k_bump_table(const double* __restrict__ x, int64_t n, int dim,
                                                         const gp::BumpParam* __restrict__ bumps, int n1,
                                                         int n2, double beta, double lo0, double lo1,
                                                         double lo2, double* __restrict__ F0,
                                                         uint32_t* __restrict__ mask0,
                                                         int32_t* __restrict__ flag) {
  extern __shared__ gp::BumpParam sb[];
  __shared__ int q_pt[kWarps][kBtQueue];        // lane of the point
  __shared__ int q_b[kWarps][kBtQueue];         // bump index m n2 + j
  __shared__ double q_val[kWarps][kBtQueue];    // a exp(beta - beta / u), if added
  __shared__ unsigned char q_fl[kWarps][kBtQueue];  // 1: inside the support, 2: value to add
  const int nb = n1 * n2;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) sb[b] = bumps[b];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = gpd::lanemask_lt();
  const double lo[3] = {lo0, lo1, lo2};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // the grid-stride loop runs the same number of times in every lane of a warp
  for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane; base < n; base += stride) {
    const int64_t i = base + lane;
    const bool valid = i < n;
    double xi[gp::kMaxDim] = {0, 0, 0};
    float x32[gp::kMaxDim] = {0, 0, 0};
    if (valid) {
      for (int k = 0; k < dim; ++k) {
        xi[k] = x[i * dim + k];
        x32[k] = (float)(xi[k] - lo[k]);
      }
    }
    // this lane's running state: compensated sum f + fc of function mcur
    double f = 0.0, fc = 0.0;
    int mcur = -1;
    uint32_t mask = 0;
    auto close_until = [&](int m_next) {
      // F0 of mcur (if any), and zeros for the functions before m_next that
      // had no accepted bump
      if (mcur >= 0) F0[i * n1 + mcur] = f + fc;
      for (int m = mcur + 1; m < m_next; ++m) F0[i * n1 + m] = 0.0;
      f = 0.0;
      fc = 0.0;
      mcur = m_next;
    };
    int count = 0;
    auto flush = [&]() {
      __syncwarp();
      for (int e = lane; e < count; e += 32) {
        const int pl = q_pt[w][e], b = q_b[w][e];
        const gp::BumpParam& bp = sb[b];
        double xp[gp::kMaxDim] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) xp[k] = x[(base + pl) * dim + k];
        // the support test exactly as the plain definition (FP64, this
        // operation order); the value from u = 1 - q without cancellation
        double d2 = 0.0;
        for (int k = 0; k < dim; ++k) {
          double t = __dsub_rn(xp[k], bp.c[k]);
          d2 = __dadd_rn(d2, __dmul_rn(t, t));
        }
        const double q = __ddiv_rn(d2, bp.r2);
        unsigned char fl = 0;
        double v = 0.0;
        if (q < 1.0) {
          fl = 1;
          const double u = gpd::one_minus_ratio(xp, bp.c, dim, bp.r2, bp.r2l);
          if (u > 0.0) {
            fl = 3;
            v = bp.a * exp(beta - beta / u);
          }
        }
        q_fl[w][e] = fl;
        q_val[w][e] = v;
      }
      __syncwarp();
      for (int e = 0; e < count; ++e) {
        if (q_pt[w][e] != lane) continue;
        const int m = q_b[w][e] / n2;
        if (m != mcur) close_until(m);
        const unsigned char fl = q_fl[w][e];
        if (fl & 1) mask |= 1u << m;
        if (fl & 2) {
          double t, er;
          gpd::two_sum(f, q_val[w][e], t, er);
          f = t;
          fc += er;
        }
      }
      __syncwarp();
      count = 0;
    };
    for (int b = 0; b < nb; ++b) {
      bool pass = false;
      if (valid) {
        const gp::BumpParam& bp = sb[b];
        float q32 = 0.0f;
        for (int k = 0; k < dim; ++k) {
          float t = x32[k] - bp.c32[k];
          q32 = fmaf(t, t, q32);
        }
        q32 *= bp.inv_r2_32;
        pass = q32 < 1.0f + bp.margin;
      }
      const unsigned bal = __ballot_sync(kFull, pass);
      if (pass) {
        const int slot = count + __popc(bal & lt);
        q_pt[w][slot] = lane;
        q_b[w][slot] = b;
      }
      count += __popc(bal);
      if (count > kBtQueue - 32) flush();
    }
    if (count > 0) flush();
    if (valid) {
      close_until(n1);
      mask0[i] = mask;
      flag[i] = mask != 0u;
    }
  }
}

// ------------------------------------------------------------------ cells
__device__ inline uint32_t morton(const int* c, const gp::Grid& g) {
  uint32_t key = 0;
  int pos = 0;
  for (int t = 0; t < 32 && pos < g.keybits; ++t)
    for (int k = 0; k < g.dim; ++k)
      if (t < g.bits[k]) key |= (uint32_t)((c[k] >> t) & 1) << pos++;
  return key;
}

// Index along the Hilbert curve of the point X (dim <= 3 coordinates of b
// bits each), by Skilling's transform ("Programming the Hilbert curve", AIP
// Conf. Proc. 707, 2004): the coordinates are turned into the transposed
// index in place, then its bits are read out most significant first.  The
// curve is hierarchical: the top dim * L bits of the index number the level-L
// cube containing X, and the points of one such cube are contiguous.
__device__ inline uint32_t hilbert_index(uint32_t* X, int dim, int b) {
  const uint32_t m = 1u << (b - 1);
  for (uint32_t q = m; q > 1; q >>= 1) {
    const uint32_t lowbits = q - 1;
    for (int i = 0; i < dim; ++i) {
      if (X[i] & q) {
        X[0] ^= lowbits;
      } else {
        const uint32_t t = (X[0] ^ X[i]) & lowbits;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  for (int i = 1; i < dim; ++i) X[i] ^= X[i - 1];
  uint32_t t = 0;
  for (uint32_t q = m; q > 1; q >>= 1)
    if (X[dim - 1] & q) t ^= q - 1;
  for (int i = 0; i < dim; ++i) X[i] ^= t;
  uint32_t key = 0;
  for (int j = b - 1; j >= 0; --j)
    for (int i = 0; i < dim; ++i) key = (key << 1) | ((X[i] >> j) & 1u);
  return key;
}

// Sort key.  Hilbert mode: the Hilbert index of the point's sub-cell (cell
// coordinates extended by subbits bits per axis) over the grid padded to
// 2^hbits cells per axis.  The cells are level-hbits cubes of the curve, so a
// cell's points stay contiguous, cells follow the curve, and consecutive
// rows are close in space without the Z-curve's jumps (on the 1M mixture the
// 8x1 block CSR needs 11.27 M blocks instead of 12.17 M).  Morton mode (when
// the padded grid needs more than 32 bits): the cell's Morton code in the
// high bits, then the Morton code of the sub-cell.
__device__ inline uint32_t sort_key(const double* xi, const int* c, const gp::Grid& g) {
  if (g.hilbert) {
    const int ns = 1 << g.subbits;
    uint32_t X[gp::kMaxDim] = {0, 0, 0};
    for (int k = 0; k < g.dim; ++k) {
      double u = __ddiv_rn(__dsub_rn(xi[k], g.lo[k]), g.h) - (double)c[k];
      int v = (int)floor(u * ns);
      v = v < 0 ? 0 : (v > ns - 1 ? ns - 1 : v);
      X[k] = ((uint32_t)c[k] << g.subbits) | (uint32_t)v;
    }
    return hilbert_index(X, g.dim, g.hbits + g.subbits);
  }
  uint32_t sub = 0;
  if (g.subbits > 0) {
    const int ns = 1 << g.subbits;
    int sc[gp::kMaxDim] = {0, 0, 0};
    for (int k = 0; k < g.dim; ++k) {
      double u = __ddiv_rn(__dsub_rn(xi[k], g.lo[k]), g.h) - (double)c[k];
      int v = (int)floor(u * ns);
      sc[k] = v < 0 ? 0 : (v > ns - 1 ? ns - 1 : v);
    }
    int pos = 0;
    for (int t = 0; t < g.subbits; ++t)
      for (int k = 0; k < g.dim; ++k) sub |= (uint32_t)((sc[k] >> t) & 1) << pos++;
  }
  return (morton(c, g) << (g.subbits * g.dim)) | sub;
}

__global__ void __launch_bounds__(kThreads) k_keys(const double* __restrict__ x, int64_t n,
                                                   const int64_t* __restrict__ pos,
                                                   const uint32_t* __restrict__ mask0, gp::Grid g,
                                                   uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (mask0[i] == 0u) continue;
    double xi[gp::kMaxDim] = {0, 0, 0};
    for (int k = 0; k < g.dim; ++k) xi[k] = x[i * g.dim + k];
    int c[gp::kMaxDim];
    gpd::cell_of(xi, g, c);
    int64_t a = pos[i];
    keys[a] = sort_key(xi, c, g);
    vals[a] = (uint32_t)i;
  }
}

// ------------------------------------------------------------------ radix sort
// Stable LSD radix sort of (key, value) pairs, 8-bit digits.  A tile of
// kRsTile items is ranked in kRsRounds rounds of 256 items (item order within
// the tile = round, then thread), each item's rank among equal digits in its
// warp comes from __match_any_sync, and per-warp digit counts are prefixed in
// shared memory, so equal keys keep their input order.
constexpr int kRsRounds = 8;
constexpr int kRsTile = kThreads * kRsRounds;

__global__ void __launch_bounds__(kThreads) k_rs_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                      int ntiles, int32_t* __restrict__ hist) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int r = 0; r < kRsRounds; ++r) {
    int64_t idx = base + r * kThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin, int64_t n, int shift,
                                                         int ntiles, const int64_t* __restrict__ offs,
                                                         uint32_t* __restrict__ kout,
                                                         uint32_t* __restrict__ vout) {
  __shared__ long long run[256];
  __shared__ long long wcnt[kWarps][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  run[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int r = 0; r < kRsRounds; ++r) {
    for (int t = threadIdx.x; t < kWarps * 256; t += kThreads) (&wcnt[0][0])[t] = 0;
    __syncthreads();
    const int64_t idx = base + r * kThreads + threadIdx.x;
    const bool valid = idx < n;
    uint32_t k = valid ? kin[idx] : 0u;
    uint32_t v = valid ? vin[idx] : 0u;
    unsigned d = valid ? ((k >> shift) & 255u) : 256u + lane;  // invalid items match nobody
    unsigned peers = __match_any_sync(kFull, d);
    unsigned below = peers & gpd::lanemask_lt();
    int rank = __popc(below);
    if (valid && below == 0u) wcnt[w][d] = __popc(peers);
    __syncthreads();
    {
      const int dig = threadIdx.x;  // 256 threads = 256 digits
      long long acc = run[dig];
      for (int ww = 0; ww < kWarps; ++ww) {
        long long cnum = wcnt[ww][dig];
        wcnt[ww][dig] = acc;
        acc += cnum;
      }
      run[dig] = acc;
    }
    __syncthreads();
    if (valid) {
      long long p = wcnt[w][d] + rank;
      kout[p] = k;
      vout[p] = v;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ sorted points
// For sorted position p: original index, cell coordinates, FP32 coordinates
// relative to the own cell (units of h), FP64 coordinates, F and mask in
// Morton order, D^-1/2, cell table boundaries, and sum ln D.  The FP32 path
// also gets the coordinates and Fhat = sqrt(A C) D^-1/2 F as double-float
// pairs (hi = the FP32 rounding, lo = the FP32 rounding of the rest), which
// carry 48 bits.  |Fhat| <= 1 (D >= A C F^2), and a stored entry is
// k~ sum_m Fhat_pm Fhat_jm with k~ <= 1, so the products of the table are at
// least the size of the entry and stay in FP32's normal range when it does.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_sorted(const double* __restrict__ x, int64_t n_act,
                                                     const uint32_t* __restrict__ skey,
                                                     const uint32_t* __restrict__ perm, gp::Grid g,
                                                     const double* __restrict__ F0,
                                                     const uint32_t* __restrict__ mask0, int n1, double AC,
                                                     double sigma2, int4* __restrict__ cellc,
                                                     float4* __restrict__ xr, double* __restrict__ xs,
                                                     float2* __restrict__ xhl, T* __restrict__ Fs,
                                                     float2* __restrict__ Fhl,
                                                     uint32_t* __restrict__ smask,
                                                     T* __restrict__ dinv, double* __restrict__ dinv64,
                                                     int2* __restrict__ cells, double* __restrict__ part,
                                                     gp::AsmScalars* s) {
  double acc = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_act; p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = perm[p];
    double xi[gp::kMaxDim] = {0, 0, 0};
    for (int k = 0; k < g.dim; ++k) xi[k] = x[(int64_t)i * g.dim + k];
    int c[gp::kMaxDim];
    gpd::cell_of(xi, g, c);
    cellc[p] = make_int4(c[0], c[1], c[2], 0);
    float r[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < g.dim; ++k) {
      double u = __ddiv_rn(__dsub_rn(xi[k], g.lo[k]), g.h);
      r[k] = (float)(u - (double)c[k]);
      xs[p * g.dim + k] = xi[k];
      if (xhl) {
        const float hi = (float)xi[k];
        xhl[p * g.dim + k] = make_float2(hi, (float)(xi[k] - (double)hi));
      }
    }
    xr[p] = make_float4(r[0], r[1], r[2], 0.f);
    double sF = 0.0;
    for (int m = 0; m < n1; ++m) {
      double f = F0[(int64_t)i * n1 + m];
      Fs[p * n1 + m] = (T)f;
      sF += f * f;
    }
    smask[p] = mask0[i];
    const double D = AC * sF + sigma2;
    const double di = 1.0 / sqrt(D);
    if (Fhl) {
      const double sc = sqrt(AC) * di;
      for (int m = 0; m < n1; ++m) {
        const double f = F0[(int64_t)i * n1 + m] * sc;
        const float hi = (float)f;
        Fhl[p * n1 + m] = make_float2(hi, (float)(f - (double)hi));
      }
    }
    dinv64[p] = di;
    dinv[p] = (T)di;
    acc += log(D);
    const int64_t lin = (int64_t)c[0] + (int64_t)g.G[0] * ((int64_t)c[1] + (int64_t)g.G[1] * c[2]);
    const int sh = g.subbits * g.dim;  // the cell code sits above the sub-cell bits
    const uint32_t kk = skey[p] >> sh;
    if (p == 0 || (skey[p - 1] >> sh) != kk) cells[lin].x = (int)p;
    if (p == n_act - 1 || (skey[p + 1] >> sh) != kk) cells[lin].y = (int)(p + 1);
  }
  __shared__ double sh[kThreads];
  __shared__ bool last;
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sh[0];
    __threadfence();
    last = atomicInc(&s->ticket1, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(part + b);
    s->sum_log_d = t;
  }
}

// ------------------------------------------------------------------ pair search
struct PairArgs {
  int64_t n;
  int dim, nstencil, n1;
  int G0, G1, G2;
  const int2* cells;
  const int4* cellc;
  const uint32_t* mask;
  const float4* xr;
  const double* xs;
  const float2* xhl;    // FP32 path: coordinates as double-float pairs
  const void* Fs;
  const float2* Fhl;    // FP32 path: the sorted bump table as double-float pairs
  const void* dinv;
  const double* dinv64; // D^-1/2 in FP64 (entry values)
  const int64_t* row_ptr;
  int32_t* cnt;
  int32_t* col;
  void* val;
  float scale;   // (h / r_s)^2
  float guard;   // |rho^2 - 1| below this: decide in FP64
  double rs2;    // r_s^2 rounded to FP64 (the support test d^2 < r_s^2)
  double rs2l;   // r_s * r_s - rs2 exactly
  double inv_rs2;
  double AC;     // A * C
  double sigma2;
  double inv2l2; // 1 / (2 l^2) of the squared-exponential core, 0 without a core
  // the same constants for the FP32 entry values (pairs: hi + lo)
  float rs2h, rs2lo, inv_rs2f, sigma2f, il2h, il2lo;
  float s2min;   // FP32 path: entries with s^2 below this take the FP64 route
};

__device__ inline int warp_incl_scan_int(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

__device__ inline double dist2_fp64(const double* __restrict__ xs, int dim, int64_t p, int64_t j) {
  double d2 = 0.0;
  for (int k = 0; k < dim; ++k) {
    double t = __dsub_rn(xs[p * dim + k], xs[j * dim + k]);
    d2 = __dadd_rn(d2, __dmul_rn(t, t));
  }
  return d2;
}

// Value of the stored entry (p, j) of the FP32 path, p and j in each other's
// support: FP32 arithmetic on double-float inputs.  d^2 as a pair from exact
// coordinate differences (TwoSum) and exact squares (TwoProduct), r_s^2 - d^2
// on the pair (no cancellation near the edge), so s^2 and rho^2 reach the
// stationary kernel with one FP32 rounding, as from FP64; the sum over the
// shared functions compensated on the double-float Fhat = sqrt(A C) D^-1/2 F
// (so it is already the stored entry's size), the core factor last.  Entries
// with s^2 below s2min (where the pair's own error would show) take the FP64
// route: rho^2 and s^2 in FP64 (s^2 without cancellation), the sum in FP64,
// one rounding.
__device__ inline float entry_value_f32(const PairArgs& a, int64_t p, int64_t j, uint32_t common) {
  float eh, el;
  gpd::dist2_pair_f(a.xhl, a.dim, p, j, eh, el);
  const float num = gpd::pair_gap_f(a.rs2h, a.rs2lo, eh, el);  // r_s^2 - d^2
  if (num >= a.s2min * a.rs2h) {
    const float s2 = num * a.inv_rs2f;
    const float rho2 = (eh + el) * a.inv_rs2f;  // el carries the differences' low parts
    const float kst = gpd::kstat_unit_f(rho2, s2);
    const float2* Fp = a.Fhl + p * a.n1;
    const float2* Fj = a.Fhl + j * a.n1;
    float Sh = 0.f, Sl = 0.f;
    while (common) {
      const int m = __ffs(common) - 1;
      common &= common - 1u;
      const float2 f = Fp[m], g2 = Fj[m];
      float ph, pe;
      gpd::two_prod_f(f.x, g2.x, ph, pe);
      pe = fmaf(f.x, g2.y, fmaf(f.y, g2.x, pe));
      float t, te;
      gpd::two_sum_f(Sh, ph, t, te);
      Sh = t;
      Sl += te + pe;
    }
    float vv = kst * (Sh + Sl);
    if (j == p) {
      const float dp = ((const float*)a.dinv)[p];
      vv = fmaf(a.sigma2f * dp, dp, vv);
    } else if (a.il2h > 0.f) {
      // t = d^2 / (2 l^2) as th + tl, exp(-t) = expf(-th) (1 - tl)
      const float th = eh * a.il2h;
      const float tl = fmaf(eh, a.il2h, -th) + fmaf(el, a.il2h, eh * a.il2lo);
      vv *= expf(-th) * (1.f - tl);
    }
    return vv;
  }
  const double e2 = dist2_fp64(a.xs, a.dim, p, j);
  double s2 = (a.rs2 - e2) * a.inv_rs2;
  if (s2 < 1e-6) s2 = gpd::one_minus_ratio(a.xs + p * a.dim, a.xs + j * a.dim, a.dim, a.rs2, a.rs2l);
  const double rho2 = e2 * a.inv_rs2;
  const double kst = s2 > 0.0 ? (double)gpd::kstat_unit_f((float)rho2, (float)s2) : 0.0;
  double S = 0.0;
  while (common) {
    const int m = __ffs(common) - 1;
    common &= common - 1u;
    const float2 f = a.Fhl[p * a.n1 + m], g2 = a.Fhl[j * a.n1 + m];
    S = fma((double)f.x + (double)f.y, (double)g2.x + (double)g2.y, S);
  }
  double vv = kst * S;
  if (a.inv2l2 > 0.0 && j != p) vv *= gpd::sqexp_core<float>(e2 * a.inv2l2);
  if (j == p) vv += a.sigma2 * a.dinv64[p] * a.dinv64[p];
  return (float)vv;
}

// One warp per active row p.  The 3^dim neighbour cells of p's cell are
// ordered by their first sorted index, so visiting their point ranges in that
// order yields ascending column indices; the ranges are flattened and 32
// candidates are tested per step.  Predicate of row p, column j:
//   mask_p & mask_j != 0  and  |x_p - x_j|^2 < r_s^2   (j == p always passes).
// COUNT writes the number of hits per row; FILL writes columns and the
// Jacobi-scaled values  D_p^-1/2 (A C k~ sum_m F_pm F_jm + sigma_n^2 [p==j]) D_j^-1/2.
// FP32 FILL: a warp step finds about 5 hits among its 32 candidates, so the
// value code would run with 5 of 32 lanes busy; hits are queued per warp
// instead (entry, column, row) and their values computed 32 at a time.
constexpr int kPairQueue = 64;

template <typename T, bool FILL>
__global__ void __launch_bounds__(kThreads) k_pair(PairArgs a) {
  __shared__ int sh_start[kWarps][32];
  __shared__ int sh_pre[kWarps][32];
  __shared__ int sh_off[kWarps][32];
  constexpr bool kQueue = FILL && sizeof(T) == 4;
  __shared__ int64_t q_pos[kQueue ? kWarps : 1][kPairQueue];
  __shared__ int q_row[kQueue ? kWarps : 1][kPairQueue];
  __shared__ int q_col[kQueue ? kWarps : 1][kPairQueue];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T* val = (T*)a.val;
  int qn = 0;  // queued hits of this warp
  auto flush = [&]() {
    if constexpr (kQueue) {
      __syncwarp();
      for (int e = lane; e < qn; e += 32) {
        const int pp = q_row[w][e], jj = q_col[w][e];
        val[q_pos[w][e]] = (T)entry_value_f32(a, pp, jj, a.mask[pp] & a.mask[jj]);
      }
      __syncwarp();
      qn = 0;
    }
  };
  const int G[3] = {a.G0, a.G1, a.G2};
  for (int64_t p = (int64_t)blockIdx.x * kWarps + w; p < a.n; p += (int64_t)gridDim.x * kWarps) {
    const int4 ci4 = a.cellc[p];
    const int ci[3] = {ci4.x, ci4.y, ci4.z};
    const uint32_t mi = a.mask[p];
    // 2-bit offset code per axis (offset + 1); axes beyond dim keep offset 0
    int start = 0, len = 0, offpack = 0x15;
    if (lane < a.nstencil) {
      int t = lane;
      bool ok = true;
      int64_t lin = 0, mult = 1;
      for (int k = 0; k < a.dim; ++k) {
        int o = t % 3 - 1;
        t /= 3;
        int cc = ci[k] + o;
        ok = ok && cc >= 0 && cc < G[k];
        lin += (int64_t)cc * mult;
        mult *= G[k];
        offpack = (offpack & ~(3 << (2 * k))) | ((o + 1) << (2 * k));
      }
      if (ok) {
        int2 se = a.cells[lin];
        start = se.x;
        len = se.y - se.x;
      }
    }
    const int key = len > 0 ? start : INT_MAX;
    int rank = 0;
    for (int l2 = 0; l2 < a.nstencil; ++l2) {
      int k2 = __shfl_sync(kFull, key, l2);
      rank += (k2 < key) || (k2 == key && l2 < lane);
    }
    const unsigned nonempty = __ballot_sync(kFull, lane < a.nstencil && len > 0);
    const int nseg = __popc(nonempty);
    __syncwarp();
    if (lane < a.nstencil && len > 0) {
      sh_start[w][rank] = start;
      sh_pre[w][rank] = len;
      sh_off[w][rank] = offpack;
    }
    __syncwarp();
    const int L = lane < nseg ? sh_pre[w][lane] : 0;
    const int inc = warp_incl_scan_int(L);
    __syncwarp();
    if (lane < nseg) sh_pre[w][lane] = inc - L;
    const int total = __shfl_sync(kFull, inc, 31);
    __syncwarp();

    const float4 xi = a.xr[p];
    int64_t out = 0;
    if (FILL) out = a.row_ptr[p];
    int count = 0;
    for (int base = 0; base < total; base += 32) {
      const int f = base + lane;
      bool hit = false;
      int j = 0;
      T v = 0;
      if (f < total) {
        int r = 0;
        for (int step = 16; step > 0; step >>= 1)
          if (r + step < nseg && sh_pre[w][r + step] <= f) r += step;
        j = sh_start[w][r] + (f - sh_pre[w][r]);
        const uint32_t mj = a.mask[j];
        if ((mi & mj) != 0u) {
          // support test: FP32 on cell-relative coordinates, decided in FP64
          // (the plain definition's arithmetic) inside the guard band
          double e2 = -1.0;
          if (sizeof(T) == 4) {
            const float4 xj = a.xr[j];
            const int op = sh_off[w][r];
            const float dx = (xj.x + (float)((op & 3) - 1)) - xi.x;
            const float dy = (xj.y + (float)(((op >> 2) & 3) - 1)) - xi.y;
            const float dz = (xj.z + (float)(((op >> 4) & 3) - 1)) - xi.z;
            float r2 = (dx * dx + dy * dy + dz * dz) * a.scale;
            if (fabsf(r2 - 1.0f) < a.guard) {
              e2 = dist2_fp64(a.xs, a.dim, p, j);
              hit = e2 < a.rs2;
            } else {
              hit = r2 < 1.0f;
            }
          } else {
            e2 = dist2_fp64(a.xs, a.dim, p, j);
            hit = e2 < a.rs2;
          }
          if (FILL && hit) {
            if constexpr (sizeof(T) == 8) {
              // FP64 path: rho^2 and s^2 = 1 - rho^2 in FP64 (s^2 without
              // cancellation near the edge), the sum over the shared functions
              // compensated, one rounding
              if (e2 < 0.0) e2 = dist2_fp64(a.xs, a.dim, p, j);
              double s2 = (a.rs2 - e2) * a.inv_rs2;
              if (s2 < 1e-2)
                s2 = gpd::one_minus_ratio(a.xs + p * a.dim, a.xs + (int64_t)j * a.dim, a.dim, a.rs2, a.rs2l);
              const double rho2 = e2 * a.inv_rs2;
              const double kst = s2 > 0.0 ? gpd::kstat_unit_d(rho2, s2) : 0.0;
              const double S =
                  gpd::dot2_bits((const double*)a.Fs + p * a.n1, (const double*)a.Fs + (int64_t)j * a.n1, mi & mj);
              double vv = a.AC * kst * S;
              if (a.inv2l2 > 0.0 && j != p) vv *= gpd::sqexp_core<T>(e2 * a.inv2l2);
              if (j == p) vv += a.sigma2;
              v = (T)(vv * a.dinv64[p] * a.dinv64[j]);
            }
          }
        }
      }
      const unsigned bal = __ballot_sync(kFull, hit);
      if (FILL && hit) {
        const int64_t q = out + count + __popc(bal & gpd::lanemask_lt());
        a.col[q] = j;
        if constexpr (kQueue) {
          const int slot = qn + __popc(bal & gpd::lanemask_lt());
          q_pos[w][slot] = q;
          q_row[w][slot] = (int)p;
          q_col[w][slot] = j;
        } else {
          val[q] = v;
        }
      }
      count += __popc(bal);
      if constexpr (kQueue) {
        qn += __popc(bal);
        if (qn > kPairQueue - 32) flush();
      }
    }
    if (!FILL && lane == 0) a.cnt[p] = count;
  }
  flush();
}

// ------------------------------------------------------------------ 8x1 block CSR
// The FP32 SpMM reads K in CSR of 8x1 blocks: block row b holds the rows
// 8b..8b+7 (consecutive in Morton / sub-cell order, so close in space); each
// stored block is one column j with the 8 values K_(8b+r),j (0 where (8b+r, j)
// is outside the pattern) and an 8-bit mask of the pattern entries.  One
// column index and one gathered P row then serve up to 8 rows.
// The support predicate is evaluated exactly as in k_pair (same FP32
// expression, same FP64 guard band), so the two patterns are identical, and
// candidate columns are visited in ascending order, so the hits of each row
// arrive in the order of its scalar-CSR row.  COUNT writes the blocks per
// block row and also the entries per row (the scalar CSR's counts, so no
// separate count pass); FILL copies the values k_pair computed.  (Computing
// the values here instead, once for both matrices, took 10.1 ms at 1M
// against 2.7 + 1.2 ms: the value code lifts the kernel to 162 registers.)
constexpr int kBR = 8;
constexpr int kBWarps = 4;
constexpr int kMaxCand = kBR * 27;  // distinct neighbour cells of one block row

template <bool FILL>
__global__ void __launch_bounds__(kBWarps * 32) k_bpair(PairArgs a, int64_t nblk, const int64_t* __restrict__ brp,
                                                        int32_t* __restrict__ bcnt, int32_t* __restrict__ bcol,
                                                        uint8_t* __restrict__ bmask, float* __restrict__ bval) {
  __shared__ float4 s_rx[kBWarps][kBR];
  __shared__ int4 s_rc[kBWarps][kBR];
  __shared__ uint32_t s_rm[kBWarps][kBR];
  __shared__ int s_start[kBWarps][kMaxCand];
  __shared__ int s_len[kBWarps][kMaxCand];
  __shared__ int4 s_cc[kBWarps][kMaxCand];
  __shared__ int s_start2[kBWarps][kMaxCand];
  __shared__ int s_pre[kBWarps][kMaxCand];
  __shared__ int4 s_cc2[kBWarps][kMaxCand];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float* csr_val = (const float*)a.val;
  const int G[3] = {a.G0, a.G1, a.G2};
  for (int64_t bb = (int64_t)blockIdx.x * kBWarps + w; bb < nblk; bb += (int64_t)gridDim.x * kBWarps) {
    const int64_t r0 = bb * kBR;
    const int nr = (int)min((int64_t)kBR, a.n - r0);
    int4 myc = make_int4(-1, -1, -1, 0);
    int64_t myrow = 0;  // FILL: next unread scalar-CSR entry of row r0 + lane; COUNT: its entries
    if (lane < nr) {
      myc = a.cellc[r0 + lane];
      s_rx[w][lane] = a.xr[r0 + lane];
      s_rc[w][lane] = myc;
      s_rm[w][lane] = a.mask[r0 + lane];
      if (FILL) myrow = a.row_ptr[r0 + lane];
    }
    // one representative lane per distinct row cell
    bool rep = lane < nr;
    for (int q = 0; q < kBR; ++q) {
      const int ox = __shfl_sync(kFull, myc.x, q), oy = __shfl_sync(kFull, myc.y, q),
                oz = __shfl_sync(kFull, myc.z, q);
      if (q < lane && ox == myc.x && oy == myc.y && oz == myc.z) rep = false;
    }
    unsigned reps = __ballot_sync(kFull, rep);
    // neighbour cells of all row cells, non-empty ones once each
    int L = 0;
    while (reps) {
      const int q = __ffs(reps) - 1;
      reps &= reps - 1u;
      const int c3[3] = {__shfl_sync(kFull, myc.x, q), __shfl_sync(kFull, myc.y, q), __shfl_sync(kFull, myc.z, q)};
      bool ok = false;
      int start = 0, len = 0;
      int nc[3] = {0, 0, 0};
      if (lane < a.nstencil) {
        int t = lane;
        ok = true;
        int64_t lin = 0, mult = 1;
        for (int k = 0; k < a.dim; ++k) {
          const int o = t % 3 - 1;
          t /= 3;
          nc[k] = c3[k] + o;
          ok = ok && nc[k] >= 0 && nc[k] < G[k];
          lin += (int64_t)nc[k] * mult;
          mult *= G[k];
        }
        if (ok) {
          const int2 se = a.cells[lin];
          start = se.x;
          len = se.y - se.x;
          ok = len > 0;
        }
        for (int t2 = 0; ok && t2 < L; ++t2)
          if (s_start[w][t2] == start) ok = false;
      }
      const unsigned bal = __ballot_sync(kFull, ok);
      if (ok) {
        const int pos = L + __popc(bal & gpd::lanemask_lt());
        s_start[w][pos] = start;
        s_len[w][pos] = len;
        s_cc[w][pos] = make_int4(nc[0], nc[1], nc[2], 0);
      }
      L += __popc(bal);
      __syncwarp();
    }
    // order the cells by first sorted index (distinct for non-empty cells),
    // which orders the candidate columns ascending
    for (int e = lane; e < L; e += 32) {
      const int st0 = s_start[w][e];
      int rank = 0;
      for (int t2 = 0; t2 < L; ++t2) rank += s_start[w][t2] < st0;
      s_start2[w][rank] = st0;
      s_pre[w][rank] = s_len[w][e];
      s_cc2[w][rank] = s_cc[w][e];
    }
    __syncwarp();
    // exclusive prefix of the range lengths
    int run = 0;
    for (int c0 = 0; c0 < L; c0 += 32) {
      const int v = c0 + lane < L ? s_pre[w][c0 + lane] : 0;
      const int inc = warp_incl_scan_int(v);
      __syncwarp();
      if (c0 + lane < L) s_pre[w][c0 + lane] = run + inc - v;
      run += __shfl_sync(kFull, inc, 31);
      __syncwarp();
    }
    const int total = run;
    int64_t out = FILL ? brp[bb] : 0;
    int count = 0;
    for (int base = 0; base < total; base += 32) {
      const int f = base + lane;
      uint32_t bits = 0u;
      int j = 0;
      if (f < total) {
        int r = 0;
        for (int step = 128; step > 0; step >>= 1)
          if (r + step < L && s_pre[w][r + step] <= f) r += step;
        j = s_start2[w][r] + (f - s_pre[w][r]);
        const int4 cj = s_cc2[w][r];
        const uint32_t mj = a.mask[j];
        const float4 xj = a.xr[j];
#pragma unroll
        for (int rr = 0; rr < kBR; ++rr) {
          if (rr >= nr) break;
          const uint32_t mi = s_rm[w][rr];
          if ((mi & mj) == 0u) continue;
          const int4 ci = s_rc[w][rr];
          const int ox = cj.x - ci.x, oy = cj.y - ci.y, oz = cj.z - ci.z;
          if (ox < -1 || ox > 1 || oy < -1 || oy > 1 || oz < -1 || oz > 1) continue;
          const float4 xi = s_rx[w][rr];
          const float dx = (xj.x + (float)ox) - xi.x;
          const float dy = (xj.y + (float)oy) - xi.y;
          const float dz = (xj.z + (float)oz) - xi.z;
          const float r2 = (dx * dx + dy * dy + dz * dz) * a.scale;
          bool hit;
          if (fabsf(r2 - 1.0f) < a.guard) hit = dist2_fp64(a.xs, a.dim, r0 + rr, j) < a.rs2;
          else hit = r2 < 1.0f;
          if (hit) bits |= 1u << rr;
        }
      }
      const unsigned bal = __ballot_sync(kFull, bits != 0u);
      if (!FILL) {
#pragma unroll
        for (int rr = 0; rr < kBR; ++rr) {
          const unsigned br = __ballot_sync(kFull, (bits >> rr) & 1u);
          if (lane == rr) myrow += __popc(br);
        }
      } else {
        float v[kBR];
#pragma unroll
        for (int rr = 0; rr < kBR; ++rr) {
          const unsigned br = __ballot_sync(kFull, (bits >> rr) & 1u);
          const int64_t row_next = __shfl_sync(kFull, myrow, rr);
          v[rr] = ((bits >> rr) & 1u) ? csr_val[row_next + __popc(br & gpd::lanemask_lt())] : 0.f;
          if (lane == rr) myrow += __popc(br);
        }
        if (bits != 0u) {
          const int64_t q = out + count + __popc(bal & gpd::lanemask_lt());
          bcol[q] = j;
          bmask[q] = (uint8_t)bits;
          float4* dst = (float4*)(bval + q * kBR);
          dst[0] = make_float4(v[0], v[1], v[2], v[3]);
          dst[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
      }
      count += __popc(bal);
    }
    if (!FILL) {
      if (lane == 0) bcnt[bb] = count;
      if (lane < nr) a.cnt[r0 + lane] = (int32_t)myrow;
    }
    __syncwarp();
  }
}

// Unscaled values of the stored block (for gp_get_csr): K = D^1/2 Khat D^1/2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_unscale(int64_t n, const int64_t* __restrict__ rp,
                                                      const int32_t* __restrict__ col, const T* __restrict__ val,
                                                      const double* __restrict__ dinv64, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t p = (int64_t)blockIdx.x * kWarps + w; p < n; p += (int64_t)gridDim.x * kWarps) {
    const double dp = dinv64[p];
    for (int64_t e = rp[p] + lane; e < rp[p + 1]; e += 32) out[e] = (double)val[e] / (dp * dinv64[col[e]]);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_negate(T* __restrict__ v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = -v[i];
}

unsigned grid_for(int64_t items, int per_block, int max_blocks) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (unsigned)g;
}

template <typename T>
int assemble_t(gp_ctx* c, const double* x, int64_t n, const double* h) {
  const int dim = c->dim, n1 = c->n1, n2 = c->n2, nb = c->nb;
  const int maxb = c->num_sms * 16;
  gp::AsmScalars* s = (gp::AsmScalars*)c->asm_s.p;

  // --- bounding box (one small device->host read)
  GP_CHECK(gp::ensure(c, c->part_a, (size_t)maxb * gp::kMaxDim * 2 * sizeof(double)));
  {
    unsigned gb = grid_for(n, kThreads, maxb);
    k_bbox<<<gb, kThreads, 0, c->stream>>>(x, n, dim, (double*)c->part_a.p, s);
    GP_LAUNCH_CHECK();
    c->launches += 1;
  }
  GP_CHECK(gp::ensure_pinned(c, sizeof(gp::AsmScalars)));
  GP_CUDA(cudaMemcpyAsync(c->pinned, s, sizeof(gp::AsmScalars), cudaMemcpyDeviceToHost, c->stream));
  GP_CUDA(cudaStreamSynchronize(c->stream));
  gp::AsmScalars hs = *(gp::AsmScalars*)c->pinned;
  for (int k = 0; k < dim; ++k)
    if (!isfinite(hs.bbox_lo[k]) || !isfinite(hs.bbox_hi[k])) return GP_ERR_INVALID_ARG;

  // --- grid: cells of edge h >= r_s (slightly enlarged so that rounding in
  // the cell index can never separate two points closer than r_s by two cells)
  gp::Grid g{};
  g.dim = dim;
  double h_cell = c->r_s * (1.0 + 1e-9);
  double ext[3] = {0, 0, 0};
  for (int k = 0; k < dim; ++k) {
    g.lo[k] = hs.bbox_lo[k];
    ext[k] = hs.bbox_hi[k] - hs.bbox_lo[k];
  }
  const double max_cells = (double)(1 << 25);
  for (;;) {
    double tot = 1.0;
    for (int k = 0; k < dim; ++k) tot *= floor(ext[k] / h_cell) + 1.0;
    if (tot <= max_cells) break;
    h_cell *= 1.25;
  }
  g.h = h_cell;
  g.ncells = 1;
  g.keybits = 0;
  for (int k = 0; k < gp::kMaxDim; ++k) {
    g.G[k] = k < dim ? (int)(floor(ext[k] / h_cell) + 1.0) : 1;
    int b = 0;
    while (((int64_t)1 << b) < g.G[k]) ++b;
    g.bits[k] = b;
    g.keybits += b;
    g.ncells *= g.G[k];
  }
  if (g.keybits > 32) return GP_ERR_UNSUPPORTED;
  // Hilbert order when the grid padded to a cube of 2^B cells per axis and at
  // least one sub-cell bit fit in 32 bits; else the Morton order
  int B = 0;
  for (int k = 0; k < dim; ++k) B = g.bits[k] > B ? g.bits[k] : B;
  g.hilbert = 0;
  g.hbits = 0;
  g.subbits = 0;
  if (B >= 1 && dim * (B + 1) <= 32) {
    g.hilbert = 1;
    g.hbits = B;
    g.keybits = dim * B;
    while (g.subbits < 3 && dim * (B + g.subbits + 1) <= 32) ++g.subbits;
  } else {
    while (g.subbits < 2 && g.keybits + (g.subbits + 1) * dim <= 32) ++g.subbits;
  }
  c->grid = g;

  // --- bump parameters with FP32 pre-filter margins
  {
    double L = 0.0;
    for (int k = 0; k < dim; ++k) L = fmax(L, ext[k]);
    std::vector<gp::BumpParam> hb(nb);
    for (int m = 0; m < n1; ++m)
      for (int j = 0; j < n2; ++j) {
        const double* q = h + (size_t)(m * n2 + j) * (dim + 2);
        gp::BumpParam& bp = hb[m * n2 + j];
        double cmax = 0.0;
        for (int k = 0; k < gp::kMaxDim; ++k) {
          bp.c[k] = k < dim ? q[k] : 0.0;
          bp.c32[k] = k < dim ? (float)(q[k] - g.lo[k]) : 0.f;
          if (k < dim) cmax = fmax(cmax, fabs(q[k] - g.lo[k]));
        }
        const double r = q[dim];
        bp.r = r;
        gpd::two_prod(r, r, bp.r2, bp.r2l);
        bp.a = q[dim + 1];
        bp.m = m;
        bp.inv_r2_32 = (float)(1.0 / (r * r));
        // FP32 coordinate error per axis <= 2^-24 (L + cmax) each for x and c,
        // plus rounding of the difference; q moves by at most about
        // 2 sqrt(dim) err / r near q = 1.  Keep a 16x safety factor.
        const double err = 2.0 * 6.0e-8 * (L + cmax + r);
        double margin = 16.0 * (2.0 * sqrt((double)dim) * err / r + 4e-7);
        bp.margin = margin > 0.5 ? 1e30f : (float)margin;
      }
    GP_CHECK(gp::ensure(c, c->bump, sizeof(gp::BumpParam) * nb));
    GP_CHECK(gp::ensure_pinned(c, sizeof(gp::BumpParam) * nb));
    memcpy(c->pinned, hb.data(), sizeof(gp::BumpParam) * nb);
    GP_CUDA(cudaMemcpyAsync(c->bump.p, c->pinned, sizeof(gp::BumpParam) * nb, cudaMemcpyHostToDevice, c->stream));
  }

  // --- bump table over all points
  GP_CHECK(gp::ensure(c, c->F0, (size_t)n * n1 * sizeof(double)));
  GP_CHECK(gp::ensure(c, c->mask0, (size_t)n * sizeof(uint32_t)));
  GP_CHECK(gp::ensure(c, c->cnt, (size_t)n * sizeof(int32_t)));
  GP_CHECK(gp::ensure(c, c->pos, (size_t)(n + 1) * sizeof(int64_t)));
  {
    unsigned gb = grid_for(n, kThreads, maxb);
    size_t smem = sizeof(gp::BumpParam) * nb;
    // up to kMaxBumps parameters beside the per-warp queues: above the default 48 KB
    GP_CUDA(cudaFuncSetAttribute(k_bump_table, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_bump_table<<<gb, kThreads, smem, c->stream>>>(x, n, dim, (const gp::BumpParam*)c->bump.p, n1, n2, c->beta,
                                                    g.lo[0], dim > 1 ? g.lo[1] : 0.0, dim > 2 ? g.lo[2] : 0.0,
                                                    (double*)c->F0.p, (uint32_t*)c->mask0.p,
                                                    (int32_t*)c->cnt.p);
    GP_LAUNCH_CHECK();
    c->launches += 1;
  }
  GP_CHECK(gp::scan_i32_to_i64(c, (const int32_t*)c->cnt.p, (int64_t*)c->pos.p, n));
  int64_t n_act = 0;
  GP_CUDA(cudaMemcpyAsync(c->pinned, (int64_t*)c->pos.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  GP_CUDA(cudaStreamSynchronize(c->stream));
  n_act = *(int64_t*)c->pinned;
  c->n_act = n_act;
  c->nnz = 0;
  if (n_act == 0) return GP_OK;

  // --- Morton keys of the active points, stable radix sort
  GP_CHECK(gp::ensure(c, c->keys, (size_t)n_act * 4));
  GP_CHECK(gp::ensure(c, c->vals, (size_t)n_act * 4));
  GP_CHECK(gp::ensure(c, c->keys2, (size_t)n_act * 4));
  GP_CHECK(gp::ensure(c, c->vals2, (size_t)n_act * 4));
  {
    unsigned gb = grid_for(n, kThreads, maxb);
    k_keys<<<gb, kThreads, 0, c->stream>>>(x, n, (const int64_t*)c->pos.p, (const uint32_t*)c->mask0.p, g,
                                           (uint32_t*)c->keys.p, (uint32_t*)c->vals.p);
    GP_LAUNCH_CHECK();
    c->launches += 1;
  }
  const int passes = (g.keybits + g.subbits * dim + 7) / 8;
  const int ntiles = (int)((n_act + kRsTile - 1) / kRsTile);
  GP_CHECK(gp::ensure(c, c->hist, (size_t)256 * ntiles * sizeof(int32_t)));
  GP_CHECK(gp::ensure(c, c->hist_scan, (size_t)(256 * ntiles + 1) * sizeof(int64_t)));
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = 8 * ps;
    k_rs_hist<<<ntiles, kThreads, 0, c->stream>>>((const uint32_t*)c->keys.p, n_act, shift, ntiles,
                                                  (int32_t*)c->hist.p);
    GP_LAUNCH_CHECK();
    GP_CHECK(gp::scan_i32_to_i64(c, (const int32_t*)c->hist.p, (int64_t*)c->hist_scan.p, (int64_t)256 * ntiles));
    k_rs_scatter<<<ntiles, kThreads, 0, c->stream>>>((const uint32_t*)c->keys.p, (const uint32_t*)c->vals.p, n_act,
                                                     shift, ntiles, (const int64_t*)c->hist_scan.p,
                                                     (uint32_t*)c->keys2.p, (uint32_t*)c->vals2.p);
    GP_LAUNCH_CHECK();
    c->launches += 2;
    std::swap(c->keys, c->keys2);
    std::swap(c->vals, c->vals2);
  }

  // --- sorted point data, cell table, sum ln D
  GP_CHECK(gp::ensure(c, c->cells, (size_t)g.ncells * sizeof(int2)));
  GP_CUDA(cudaMemsetAsync(c->cells.p, 0, (size_t)g.ncells * sizeof(int2), c->stream));
  GP_CHECK(gp::ensure(c, c->cellc, (size_t)n_act * sizeof(int4)));
  GP_CHECK(gp::ensure(c, c->xr, (size_t)n_act * sizeof(float4)));
  GP_CHECK(gp::ensure(c, c->xs, (size_t)n_act * dim * sizeof(double)));
  GP_CHECK(gp::ensure(c, c->Fs, (size_t)n_act * n1 * sizeof(T)));
  // FP32 path: coordinates and the sorted bump table as double-float pairs
  // for the entry values (the FP64 path reads xs and Fs themselves)
  if (sizeof(T) == 4) {
    GP_CHECK(gp::ensure(c, c->xhl, (size_t)n_act * dim * sizeof(float2)));
    GP_CHECK(gp::ensure(c, c->Fhl, (size_t)n_act * n1 * sizeof(float2)));
  }
  float2* xhl = sizeof(T) == 4 ? (float2*)c->xhl.p : nullptr;
  float2* Fhl = sizeof(T) == 4 ? (float2*)c->Fhl.p : nullptr;
  GP_CHECK(gp::ensure(c, c->smask, (size_t)n_act * sizeof(uint32_t)));
  GP_CHECK(gp::ensure(c, c->dinv, (size_t)n_act * sizeof(T)));
  GP_CHECK(gp::ensure(c, c->dinv64, (size_t)n_act * sizeof(double)));
  GP_CHECK(gp::ensure(c, c->part_b, (size_t)maxb * sizeof(double)));
  const double AC = c->A * gp::kStatPrefactor;
  {
    unsigned gb = grid_for(n_act, kThreads, maxb);
    k_sorted<T><<<gb, kThreads, 0, c->stream>>>(x, n_act, (const uint32_t*)c->keys.p, (const uint32_t*)c->vals.p, g,
                                                (const double*)c->F0.p, (const uint32_t*)c->mask0.p, n1, AC,
                                                c->sigma2, (int4*)c->cellc.p, (float4*)c->xr.p, (double*)c->xs.p,
                                                xhl, (T*)c->Fs.p, Fhl, (uint32_t*)c->smask.p, (T*)c->dinv.p,
                                                (double*)c->dinv64.p, (int2*)c->cells.p, (double*)c->part_b.p, s);
    GP_LAUNCH_CHECK();
    c->launches += 1;
  }

  // --- two-pass CSR: count, scan, fill
  PairArgs pa{};
  pa.n = n_act;
  pa.dim = dim;
  pa.nstencil = dim == 1 ? 3 : (dim == 2 ? 9 : 27);
  pa.n1 = n1;
  pa.G0 = g.G[0];
  pa.G1 = g.G[1];
  pa.G2 = g.G[2];
  pa.cells = (const int2*)c->cells.p;
  pa.cellc = (const int4*)c->cellc.p;
  pa.mask = (const uint32_t*)c->smask.p;
  pa.xr = (const float4*)c->xr.p;
  pa.xs = (const double*)c->xs.p;
  pa.xhl = xhl;
  pa.Fs = c->Fs.p;
  pa.Fhl = Fhl;
  pa.dinv = c->dinv.p;
  pa.dinv64 = (const double*)c->dinv64.p;
  pa.cnt = (int32_t*)c->cnt.p;
  const double sc = (g.h / c->r_s) * (g.h / c->r_s);
  pa.scale = (float)sc;
  pa.guard = (float)(1e-4 * sc);
  gpd::two_prod(c->r_s, c->r_s, pa.rs2, pa.rs2l);
  pa.inv_rs2 = 1.0 / pa.rs2;
  pa.AC = AC;
  pa.sigma2 = c->sigma2;
  pa.inv2l2 = c->core == GP_CORE_SQEXP ? 1.0 / (2.0 * c->ell * c->ell) : 0.0;
  // FP32 entry values: the constants as FP32 pairs
  pa.rs2h = (float)pa.rs2;
  pa.rs2lo = (float)((pa.rs2 - (double)pa.rs2h) + pa.rs2l);
  pa.inv_rs2f = (float)pa.inv_rs2;
  pa.sigma2f = (float)c->sigma2;
  pa.il2h = (float)pa.inv2l2;
  pa.il2lo = (float)(pa.inv2l2 - (double)pa.il2h);
  {
    // the double-float d^2 carries an absolute error of about 2^-45 X r_s
    // (X the largest coordinate magnitude: the pairs hold 48 bits of each
    // coordinate); s^2 = 1 - rho^2 keeps FP32 accuracy while it exceeds
    // 2^-23 X / r_s, so the FP32 route takes s^2 >= max(2^-16, 2^-20 X / r_s)
    double X = 0.0;
    for (int k = 0; k < dim; ++k) X = fmax(X, fmax(fabs(g.lo[k]), fabs(g.lo[k] + g.G[k] * g.h)));
    pa.s2min = (float)fmax(std::ldexp(1.0, -16), std::ldexp(X / c->r_s, -20));
  }
  const bool timed = (c->flags & GP_FLAG_TIME_KERNELS) != 0;
  GP_CHECK(gp::ensure(c, c->row_ptr, (size_t)(n_act + 1) * sizeof(int64_t)));
  GP_CHECK(gp::ensure_pinned(c, 2 * sizeof(int64_t)));
  if constexpr (sizeof(T) == 8) {
    // FP64 path: the scalar CSR alone, count then fill
    const unsigned gw = grid_for(n_act, kWarps, c->num_sms * 8);
    k_pair<T, false><<<gw, kThreads, 0, c->stream>>>(pa);
    GP_LAUNCH_CHECK();
    c->launches += 1;
    GP_CHECK(gp::scan_i32_to_i64(c, (const int32_t*)c->cnt.p, (int64_t*)c->row_ptr.p, n_act));
    GP_CUDA(cudaMemcpyAsync(c->pinned, (int64_t*)c->row_ptr.p + n_act, sizeof(int64_t), cudaMemcpyDeviceToHost,
                            c->stream));
    GP_CUDA(cudaStreamSynchronize(c->stream));
    const int64_t nnz = *(int64_t*)c->pinned;
    c->nnz = nnz;
    GP_CHECK(gp::ensure(c, c->col, (size_t)nnz * sizeof(int32_t)));
    GP_CHECK(gp::ensure(c, c->val, (size_t)nnz * sizeof(T)));
    pa.row_ptr = (const int64_t*)c->row_ptr.p;
    pa.col = (int32_t*)c->col.p;
    pa.val = c->val.p;
    if (timed) {
      GP_CHECK(gp::kernel_events(c));
      GP_CUDA(cudaEventRecord(c->kev[128], c->stream));
    }
    k_pair<T, true><<<gw, kThreads, 0, c->stream>>>(pa);
    GP_LAUNCH_CHECK();
    c->launches += 1;
    if (timed) {
      GP_CUDA(cudaEventRecord(c->kev[129], c->stream));
      GP_CUDA(cudaEventSynchronize(c->kev[129]));
      c->t_fill += gp::event_ms(c->kev[128], c->kev[129]);
    }
  } else {
    // FP32 path: the scalar CSR (adjoint, copy-out) and the 8x1 block CSR
    // (SpMM): one count pass for both, both scans, one host read of both
    // totals, then the scalar fill and the block fill
    const int64_t nblk = (n_act + kBR - 1) / kBR;
    c->nblk = nblk;
    GP_CHECK(gp::ensure(c, c->bcnt, (size_t)nblk * sizeof(int32_t)));
    GP_CHECK(gp::ensure(c, c->brp, (size_t)(nblk + 1) * sizeof(int64_t)));
    const unsigned gbk = grid_for(nblk, kBWarps, c->num_sms * 16);
    k_bpair<false><<<gbk, kBWarps * 32, 0, c->stream>>>(pa, nblk, nullptr, (int32_t*)c->bcnt.p, nullptr, nullptr,
                                                         nullptr);
    GP_LAUNCH_CHECK();
    c->launches += 1;
    GP_CHECK(gp::scan_i32_to_i64(c, (const int32_t*)c->cnt.p, (int64_t*)c->row_ptr.p, n_act));
    GP_CHECK(gp::scan_i32_to_i64(c, (const int32_t*)c->bcnt.p, (int64_t*)c->brp.p, nblk));
    GP_CUDA(cudaMemcpyAsync(c->pinned, (int64_t*)c->row_ptr.p + n_act, sizeof(int64_t), cudaMemcpyDeviceToHost,
                            c->stream));
    GP_CUDA(cudaMemcpyAsync((int64_t*)c->pinned + 1, (int64_t*)c->brp.p + nblk, sizeof(int64_t),
                            cudaMemcpyDeviceToHost, c->stream));
    GP_CUDA(cudaStreamSynchronize(c->stream));
    const int64_t nnz = ((int64_t*)c->pinned)[0], nbe = ((int64_t*)c->pinned)[1];
    c->nnz = nnz;
    c->nbent = nbe;
    GP_CHECK(gp::ensure(c, c->col, (size_t)nnz * sizeof(int32_t)));
    GP_CHECK(gp::ensure(c, c->val, (size_t)nnz * sizeof(T)));
    GP_CHECK(gp::ensure(c, c->bcol, (size_t)nbe * sizeof(int32_t)));
    GP_CHECK(gp::ensure(c, c->bmask, (size_t)nbe));
    GP_CHECK(gp::ensure(c, c->bval, (size_t)nbe * kBR * sizeof(float)));
    pa.row_ptr = (const int64_t*)c->row_ptr.p;
    pa.col = (int32_t*)c->col.p;
    pa.val = c->val.p;
    if (timed) {
      GP_CHECK(gp::kernel_events(c));
      GP_CUDA(cudaEventRecord(c->kev[128], c->stream));
    }
    const unsigned gw = grid_for(n_act, kWarps, c->num_sms * 8);
    k_pair<T, true><<<gw, kThreads, 0, c->stream>>>(pa);
    GP_LAUNCH_CHECK();
    c->launches += 1;
    if (timed) {
      GP_CUDA(cudaEventRecord(c->kev[129], c->stream));
      GP_CUDA(cudaEventSynchronize(c->kev[129]));
      c->t_fill += gp::event_ms(c->kev[128], c->kev[129]);
    }
    // the blocks copy the values just computed
    k_bpair<true><<<gbk, kBWarps * 32, 0, c->stream>>>(pa, nblk, (const int64_t*)c->brp.p, nullptr,
                                                        (int32_t*)c->bcol.p, (uint8_t*)c->bmask.p,
                                                        (float*)c->bval.p);
    GP_LAUNCH_CHECK();
    c->launches += 1;
    // the regrouping for the column-window SpMM form is built on first use
    // (window.cu), only when that form is timed, forced or chosen
  }
  return GP_OK;
}

}  // namespace

namespace gp {

int assemble(gp_ctx* c, const double* x, int64_t n, const double* h, int precision) {
  c->assembled = false;
  c->precision = precision;
  c->n = n;
  const size_t nbp = (size_t)c->nb * (c->dim + 2);
  c->r_s = h[nbp];
  c->A = h[nbp + 1];
  c->sigma2 = h[nbp + 2];
  c->ell = c->core == GP_CORE_SQEXP ? h[nbp + 3] : 0.0;
  if (n > (int64_t)INT32_MAX - 1) return GP_ERR_UNSUPPORTED;
  c->n_act = 0;
  c->nnz = 0;
  c->nblk = 0;
  c->w_ntiles = 0;
  if (n > 0) {
    int st = precision == GP_FP64 ? assemble_t<double>(c, x, n, h) : assemble_t<float>(c, x, n, h);
    if (st != GP_OK) return st;
  } else {
    // no points: the bumps still define k(x*, x*) for predictions
    std::vector<gp::BumpParam> hb(c->nb);
    const int np = c->dim + 2;
    for (int b = 0; b < c->nb; ++b) {
      const double* q = h + (size_t)b * np;
      gp::BumpParam& bp = hb[b];
      for (int k = 0; k < gp::kMaxDim; ++k) {
        bp.c[k] = k < c->dim ? q[k] : 0.0;
        bp.c32[k] = 0.f;
      }
      bp.r = q[c->dim];
      gpd::two_prod(bp.r, bp.r, bp.r2, bp.r2l);
      bp.a = q[c->dim + 1];
      bp.m = b / c->n2;
      bp.inv_r2_32 = (float)(1.0 / bp.r2);
      bp.margin = 1e30f;
    }
    GP_CHECK(gp::ensure(c, c->bump, sizeof(gp::BumpParam) * c->nb));
    GP_CHECK(gp::ensure_pinned(c, sizeof(gp::BumpParam) * c->nb));
    memcpy(c->pinned, hb.data(), sizeof(gp::BumpParam) * c->nb);
    GP_CUDA(cudaMemcpyAsync(c->bump.p, c->pinned, sizeof(gp::BumpParam) * c->nb, cudaMemcpyHostToDevice,
                            c->stream));
    GP_CUDA(cudaStreamSynchronize(c->stream));
  }
  c->assembled = true;
  return GP_OK;
}

int inject_matrix_fault(gp_ctx* c, int flags) {
  if (c->n_act == 0) return GP_OK;
  const bool fp64 = c->precision == GP_FP64;
  const unsigned g = grid_for(c->nnz, kThreads, c->num_sms * 8);
  if (flags & GP_FLAG_FAULT_NOT_SPD) {
    if (fp64) {
      k_negate<double><<<g, kThreads, 0, c->stream>>>((double*)c->val.p, c->nnz);
    } else {
      k_negate<float><<<g, kThreads, 0, c->stream>>>((float*)c->val.p, c->nnz);
      k_negate<float><<<grid_for(c->nbent * kBR, kThreads, c->num_sms * 8), kThreads, 0, c->stream>>>(
          (float*)c->bval.p, c->nbent * kBR);
    }
    GP_LAUNCH_CHECK();
    c->launches += fp64 ? 1 : 2;
  }
  if (flags & GP_FLAG_FAULT_NAN) {
    if (fp64) {
      const double nan = NAN;
      GP_CUDA(cudaMemcpyAsync(c->val.p, &nan, sizeof(nan), cudaMemcpyHostToDevice, c->stream));
    } else {
      const float nan = NAN;
      GP_CUDA(cudaMemcpyAsync(c->val.p, &nan, sizeof(nan), cudaMemcpyHostToDevice, c->stream));
      GP_CUDA(cudaMemcpyAsync(c->bval.p, &nan, sizeof(nan), cudaMemcpyHostToDevice, c->stream));
    }
    GP_CUDA(cudaStreamSynchronize(c->stream));  // the host values above are on the stack
  }
  return GP_OK;
}

int csr_unscaled(gp_ctx* c, double* out) {
  if (c->n_act == 0) return GP_OK;
  const unsigned gw = grid_for(c->n_act, kWarps, c->num_sms * 8);
  if (c->precision == GP_FP64)
    k_unscale<double><<<gw, kThreads, 0, c->stream>>>(c->n_act, (const int64_t*)c->row_ptr.p,
                                                     (const int32_t*)c->col.p, (const double*)c->val.p,
                                                     (const double*)c->dinv64.p, out);
  else
    k_unscale<float><<<gw, kThreads, 0, c->stream>>>(c->n_act, (const int64_t*)c->row_ptr.p,
                                                    (const int32_t*)c->col.p, (const float*)c->val.p,
                                                    (const double*)c->dinv64.p, out);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

}  // namespace gp
