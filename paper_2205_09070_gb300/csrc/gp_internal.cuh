// Internal declarations shared by the translation units of libgpsparse.
// Paper: arXiv 2205.09070 (sparse exact GPs with compactly supported,
// non-stationary bump-sum kernels).  Section / equation references below are
// to that paper.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <vector>

#include "../../include/gpsparse.h"

namespace gp {

constexpr int kMaxDim = 3;
constexpr int kMaxFuncs = 32;      // support mask is one 32-bit word
constexpr int kMaxBumps = 512;     // n_funcs * n_bumps
constexpr int kMaxProbes = 64;     // probe sign bits: two 32-bit words per row
constexpr int kMaxCols = 68;       // 1 + n_probes, padded to a multiple of 4
constexpr int kMaxLanczos = 64;
constexpr int kScanItems = 4096;   // elements per block of the 3-phase scan
constexpr double kStatPrefactor = 0.26596152026762182;  // sqrt(2) / (3 sqrt(pi)) = k~(0), Eq. eq:kstat

// One bump of Eq. eq:bump, in the layout the kernels read.
struct BumpParam {
  double c[kMaxDim];   // centre
  double r2;           // radius^2
  double a;            // amplitude
  double r;            // radius
  double r2l;          // radius^2 - r2 exactly (r2 + r2l = radius * radius)
  float c32[kMaxDim];  // centre - lo, FP32 (for the pre-filter)
  float inv_r2_32;     // 1 / r^2, FP32
  float margin;        // pre-filter accepts q32 < 1 + margin, then re-tests in FP64
  int m;               // function index
};

// Uniform search grid (cells of edge h >= r_s, Morton-ordered).
struct Grid {
  double lo[kMaxDim];
  double h;          // cell edge
  int G[kMaxDim];    // cells per dimension
  int bits[kMaxDim]; // Morton bits per dimension
  int dim;
  int keybits;       // bits of the cell Morton code
  int subbits;       // bits per axis of the sub-cell order inside a cell
  int hilbert;       // 1: points follow a Hilbert curve over the cells padded to 2^hbits per
                     // axis and their sub-cells; 0: the Morton (Z) order
  int hbits;         // bits per axis of the cell part of the Hilbert index
  int64_t ncells;
};

// Scalars of one batched CG run, in device memory.
struct CgState {
  double rr[kMaxCols];
  double rr0[kMaxCols];
  double alpha[kMaxCols];
  double beta[kMaxCols];
  int done[kMaxCols];
  int steps[kMaxCols];     // Lanczos steps recorded per column
  int iter;                // iterations completed
  int finished;            // set by the last kernel of an iteration: later kernels return at once
  int pending;             // all columns converged / breakdown / cap, seen by the iteration's first update
  int status;              // GP_OK or GP_ERR_NOT_SPD
  int bad_col;
  unsigned ticket_a;       // last-block tickets (reset by the last block)
  unsigned run_cnt;        // columns still running after this iteration (reset by the last block)
  unsigned ticket_b;
  unsigned ticket_c;
  int max_iter;
  double tol2;             // cg_rtol^2
  // FP32 batched path: iteration-parity copies, so that one block of a
  // kernel can publish iteration t+1 while the others still read iteration t
  double rrp[2][kMaxCols];   // rho = r^T M^-1 r (= |r|^2 without preconditioning)
  double crr[2][kMaxCols];   // |r|^2, for the convergence test
  int donep[2][kMaxCols];
  int fin[2];
};

// Reductions produced by assembly / likelihood kernels.
struct AsmScalars {
  double bbox_lo[kMaxDim];
  double bbox_hi[kMaxDim];
  double sum_log_d;        // sum over active rows of ln K_ii
  double inact_y2;         // sum over inactive rows of y_i^2
  long long n_inactive;
  double quad_form;        // y_act^T alpha_act
  double slq_mean;         // mean over probes of the Lanczos quadrature (already x N_act)
  double slq_var;          // sample variance of the probe terms
  double grad_A;
  double grad_rs;
  double grad_s2;
  double grad_l;           // core length scale (GP_CORE_SQEXP)
  unsigned ticket0;
  unsigned ticket1;
  unsigned ticket2;
  unsigned ticket3;
  unsigned ticket4;
  unsigned ticket5;
  int status;
  int pc_status;           // GP_ERR_NOT_SPD if a diagonal block failed to factor
};

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

// One way of running Q = Khat P (spmm.cu): the kernel, its launch shape and,
// for the TMA forms, the tensor map of P (an opaque 128-byte CUtensorMap).
struct SpmmPlan {
  int variant = -1;  // GP_SPMM_*
  int kp = 0;
  const void* fn = nullptr;
  size_t smem = 0;
  unsigned grid = 0;
  int stages = 0;            // GP_SPMM_WINDOW: shared-memory stages of the segment ring
  bool fused_alpha = false;  // the product also forms the CG step alpha (its last CTA)
  int k = 0, m_hist = 0;     // columns of the run and Lanczos steps recorded (fused alpha)
  alignas(64) unsigned char tmap[128] = {};
};

// Grouped CG launches: the CG runs of many independent GPs advanced by the
// same launches.  A CTA of a grouped launch works for one instance exactly as
// the CTA of the same index in that instance's own launch would, so each
// instance computes what a run on its own computes.
enum GroupKind { kGSpmm = 0, kGPc = 1, kGUpd = 2, kGUpdR = 3 };
struct GInst {
  int64_t n, nblk;  // active rows, 8-row block rows
  const int64_t* brp;
  const int32_t* bcol;
  const float4* bval;
  float4 *X, *R, *P, *Q, *Z;
  const float4* D;  // what the X, P update adds: Z when preconditioned, else R
  const float* Minv;
  double *part_a, *part_b, *hist_alpha, *hist_beta;
  CgState* st;
  int grid[4];  // the instance's own grid size per GroupKind
};
// inst == nullptr: an ordinary launch for one GP with its own arguments.
// Otherwise CTA b works for instance map[b] >> kGroupShift as its CTA
// map[b] & kGroupMask (for the per-column kernels, the column).
struct Group {
  const GInst* inst;
  const uint32_t* map;
};
constexpr int kGroupShift = 20;
constexpr uint32_t kGroupMask = (1u << kGroupShift) - 1u;
constexpr int kMaxGroup = 1 << (32 - kGroupShift);  // instances per grouped launch

}  // namespace gp

struct gp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int dim = 0, n1 = 0, n2 = 0, nb = 0;
  double beta = 1.0;
  int core = GP_CORE_NONE;
  int num_sms = 0;

  // last assembly
  bool assembled = false;
  int precision = GP_FP32_MIXED;
  int64_t n = 0, n_act = 0, nnz = 0;
  double r_s = 0, A = 0, sigma2 = 0;
  double ell = 0;  // core length scale (GP_CORE_SQEXP), else 0
  gp::Grid grid{};

  // device buffers (grow-only)
  gp::DevBuf x_in, y_in, out_tmp;
  gp::DevBuf xstar_in, pred_tmp;  // gp_predict: staged test points, posterior means
  gp::DevBuf pv_B, pv_prior;      // gp_predict_var: right-hand-side block, prior variances
  gp::DevBuf grp_inst, grp_map;   // grouped CG launches: instance table, per-CTA maps
  gp::DevBuf taylor;              // scalars of the truncated-Taylor log-determinant
  gp::DevBuf bump;
  gp::DevBuf mask0, F0, pos;
  gp::DevBuf keys, vals, keys2, vals2, hist, hist_scan, scan_part;
  gp::DevBuf cells;
  gp::DevBuf perm, skey, cellc, xr, xs, xhl, Fs, Fhl, smask, dinv, dinv64;
  gp::DevBuf cnt, row_ptr, col, val;
  // 8x1 block CSR of the FP32 path (rows 8b..8b+7 per block row)
  gp::DevBuf bcnt, brp, bcol, bmask, bval;
  int64_t nblk = 0, nbent = 0;
  // the same blocks regrouped for GP_SPMM_WINDOW (window.cu): per tile of
  // block rows its segments (descriptors), the segments' runs of P rows and
  // their records (block counts, positions, values); per-tile counts and the
  // scans of those counts
  gp::DevBuf w_cnt, w_tseg, w_trun, w_trec, w_segd, w_runs, w_rec;
  int64_t w_ntiles = 0, w_nseg = 0, w_nrun = 0;
  // block-Jacobi preconditioner (FP32 path): M^-1 per block of pc_block rows
  // (FP32, pc_block^2 each); Z = M^-1 R of the preconditioned CG
  gp::DevBuf pc_Minv, pc_part, Z;
  int pc_block = 0;
  int64_t pc_nblk = 0;
  gp::DevBuf X, R, P, Q, zbits;
  gp::DevBuf part_a, part_b, part_c, hist_alpha, hist_beta;
  gp::DevBuf g, grad_part, grad_bump;
  gp::DevBuf cg, asm_s;
  gp::DevBuf csr_tmp, slq_g;

  // pinned host staging
  void* pinned = nullptr;
  size_t pinned_cap = 0;

  cudaEvent_t ev[8] = {};

  // instrumentation (GP_FLAG_TIME_KERNELS)
  int flags = 0;
  int64_t launches = 0;
  cudaEvent_t kev[2 * 64 + 4] = {};
  bool kev_ready = false;
  double t_spmm = 0.0, t_fill = 0.0, t_adj = 0.0;
  int n_spmm = 0;
  int bad_col = -1, bad_iter = 0;   // where the last CG run stopped on a breakdown
  int spmm_variant = -1;            // SpMM form of the last FP32 CG run (GP_SPMM_*)
  // CUDA graphs of one check interval of the FP32 CG loop (slot 0: plain CG,
  // slot 1: preconditioned), reused while every launch argument is the same;
  // captured on a private stream (capture is not allowed on the legacy
  // default stream) and launched on `stream`
  struct CgGraph {
    cudaGraphExec_t exec = nullptr;
    uint64_t key[48] = {};
  } cg_graph[2];
  cudaStream_t cap_stream = nullptr;
  // side stream for work that overlaps the CG loop (the SLQ eigen-solves):
  // fork / join events, and the Lanczos step counts it reads
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t aux_ev[2] = {};
  bool slq_pending = false;
  gp::DevBuf slq_steps;
  // gp_lml_grad_batched workers: contexts of their own (stream, workspace,
  // graphs), created on first use and destroyed with this context
  std::vector<gp_ctx*> workers;
  cudaStream_t owned_stream = nullptr;  // a worker's stream (0 for user contexts)
};

namespace gp {

// ---------------------------------------------------------------- host utils
int ensure(gp_ctx* c, DevBuf& b, size_t bytes);
int ensure_pinned(gp_ctx* c, size_t bytes);
int kernel_events(gp_ctx* c);            // create the timing event pool once
double event_ms(cudaEvent_t a, cudaEvent_t b);
int cuda_status(cudaError_t e);
bool is_device_ptr(const void* p);

// ---------------------------------------------------------------- launchers
// scan.cu: exclusive scan of n int32 values into int64 (out has n+1 entries,
// out[n] = total).  Deterministic 3-phase scan.
int scan_i32_to_i64(gp_ctx* c, const int32_t* in, int64_t* out, int64_t n);

// assemble.cu
int assemble(gp_ctx* c, const double* x_dev, int64_t n, const double* h, int precision);
// GP_FLAG_FAULT_NOT_SPD: negate the stored matrix (scalar and block CSR);
// GP_FLAG_FAULT_NAN: a NaN in the first stored entry (both forms)
int inject_matrix_fault(gp_ctx* c, int flags);

// precond.cu: inverses of the diagonal blocks of the assembled Khat
// (pc_block rows per block, FP32 path only); pc_block == 0 switches it off.
int precond_setup(gp_ctx* c, int pc_block);
int csr_unscaled(gp_ctx* c, double* val_out_dev);

// solve.cu (cg_run: FP32 batched CG on the 8x1 block CSR)
// warm: keep X from the previous run on the same block and start from the
// residual B - Khat X (one extra product) instead of X = 0.  rhs: solve
// Khat X = rhs for a caller-given N_act x kp FP32 block (row-major) instead of
// [yhat, probes] (then nv = 0, lanczos_steps = 0, no warm start).
int cg_run(gp_ctx* c, int k, int kp, const double* y_dev, int n_probes, uint64_t seed,
           int lanczos_steps, int max_iter, double rtol, int check_every,
           int* iters_out, double* max_rel_resid, bool use_pc, bool warm = false,
           const float* rhs = nullptr);
// The CG runs of nc GPs (contexts cs, each assembled, with its own stream) as
// one: every context is prepared as cg_run prepares it, then the iterations
// of all of them run as grouped launches on the owner's stream (an instance
// leaves the group when its run finishes), then each is read as cg_run reads
// it.  The product is the cp.async form, wide where kp allows, for every
// instance.  ys[i]: context i's targets; iters, max_rel, status: per context.
int cg_run_group(gp_ctx* owner, gp_ctx* const* cs, int nc, int k, int kp, const double* const* ys, int n_probes,
                 uint64_t seed, int lanczos_steps, int max_iter, double rtol, int check_every, bool use_pc,
                 bool warm, int* iters, double* max_rel, int* status);
// rhs: k columns of N_act doubles each (column-major) instead of [yhat, probes]
int cg_run_fp64(gp_ctx* c, int k, const double* y_dev, int n_probes, uint64_t seed,
                int lanczos_steps, int max_iter, double rtol, int check_every,
                int* iters_out, double* max_rel_resid, const double* rhs = nullptr);
int inactive_terms(gp_ctx* c, const double* y_dev);
int quad_form(gp_ctx* c, const double* y_dev, int kp);
// SLQ terms from the recorded Lanczos coefficients; with overlap the eigen-
// solves run on the context's side stream, and slq_join orders the context
// stream after them (every caller joins before it returns).
int slq(gp_ctx* c, int n_probes, int kcols, bool overlap = false);
int slq_join(gp_ctx* c);
int alpha_out(gp_ctx* c, const double* y_dev, double* alpha_dev, int kp);

// adjoint.cu
int adjoint(gp_ctx* c, int n_probes, int kp);

// logdet.cu: ln|Khat| by the truncated Taylor series of ln(I - C) with the
// probes of the last FP32 CG run (m terms); fills the SLQ scalars' slots.
int taylor_logdet(gp_ctx* c, int n_probes, int kp, int m);

// predict.cu: posterior mean at ns test points (device arrays) from alpha =
// K^-1 y in original point order (device, c->n doubles), over the last assembly.
int predict_mean(gp_ctx* c, const double* xstar, int64_t ns, const double* alpha, double* mean);
// posterior variance k(x*, x*) - kappa^T K^-1 kappa at ns test points (device
// arrays), by blocks of test points solved as right-hand-side blocks
int predict_var(gp_ctx* c, const double* xstar, int64_t ns, double* var, const gp_opts* o, int* iters_out,
                double* max_rel);

// spmm.cu: Q = Khat P on the 8x1 block CSR (c->brp, bcol, bval; P, Q, part_a
// of the context), one launch per CG iteration.
bool spmm_available(int variant, int kp);
int spmm_plan(gp_ctx* c, int kp, int variant, SpmmPlan* plan);
// the form forced by GP_FLAG_SPMM_* in flags, else the autotuner's choice for
// this matrix shape (timed once per process, needs the CG state of iteration
// 0); k columns of the run and m_hist recorded Lanczos steps, for the forms
// that also form alpha
int spmm_select(gp_ctx* c, int kp, int flags, CgState* st, SpmmPlan* plan, int k, int m_hist);
void spmm_launch(const SpmmPlan& plan, cudaStream_t s, gp_ctx* c, CgState* st);
// window.cu: the column-window form (GP_SPMM_WINDOW): regrouping of the 8x1
// block CSR built by the assembly, and the product itself (which also forms
// alpha in its last CTA)
int window_build(gp_ctx* c);
bool window_available(gp_ctx* c, int kp);
int window_plan(gp_ctx* c, int kp, SpmmPlan* plan);
void window_launch(const SpmmPlan& plan, cudaStream_t s, gp_ctx* c, CgState* st, int k, int m_hist);
// the same product with another input / output block (cp.async forms only:
// the TMA forms carry a tensor map of P)
void spmm_launch_io(const SpmmPlan& plan, cudaStream_t s, gp_ctx* c, CgState* st, const float* in, float* out);
// a grouped launch of a cp.async form (total CTAs over all instances)
void spmm_launch_group(const SpmmPlan& plan, cudaStream_t s, unsigned total, Group g);

}  // namespace gp

// ---------------------------------------------------------------- device utils
namespace gpd {

// A grouped launch (gp::Group): this CTA's instance, and its index bx in that
// instance's own grid of gx CTAs for launches of the given kind.
__device__ __forceinline__ const gp::GInst* group_cta(const gp::Group& g, int kind, int& bx, int& gx) {
  const uint32_t m = __ldg(g.map + blockIdx.x);
  const gp::GInst* I = g.inst + (m >> gp::kGroupShift);
  bx = (int)(m & gp::kGroupMask);
  gx = I->grid[kind];
  return I;
}

// Cell of a point in the uniform search grid: floor((x - lo) / h) per axis,
// clamped to the grid (a point outside it lands in a boundary cell; the exact
// distance test still decides every pair).
__device__ inline void cell_of(const double* xi, const gp::Grid& g, int* c) {
  for (int k = 0; k < gp::kMaxDim; ++k) c[k] = 0;
  for (int k = 0; k < g.dim; ++k) {
    double u = __ddiv_rn(__dsub_rn(xi[k], g.lo[k]), g.h);
    if (!(u >= 0.0)) u = 0.0;  // also NaN
    if (u > (double)(g.G[k] - 1)) u = (double)(g.G[k] - 1);
    c[k] = (int)floor(u);
  }
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the k-th output of the
// stream whose state starts at `seed` is the finaliser applied to
// seed + (k + 1) * 0x9E3779B97F4A7C15.
__host__ __device__ inline uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Rademacher sign bit of probe l at original point index i: 1 means -1.
__device__ inline unsigned probe_bit(uint64_t seed, int l, long long i) {
  return (unsigned)(splitmix64(seed, ((uint64_t)l << 40) + (uint64_t)i) >> 63);
}

// Stationary kernel of Eq. eq:kstat divided by its prefactor C = sqrt(2)/(3 sqrt(pi)),
// as a function of rho^2 = (d/r)^2 and s^2 = 1 - rho^2 (both given, s2 > 0).
// With s = sqrt(1 - rho^2) the printed form is
//   (1 + 2 rho^2) s - 3 rho^2 log((1 + s) / rho)
// and, expanding atanh(s) = log((1+s)/rho), it equals the all-positive series
//   s^5 * sum_{k>=0} 6 s^(2k) / ((2k+3)(2k+5)),
// which is free of the cancellation the printed form suffers as rho -> 1.
__device__ inline float kstat_unit_f(float rho2, float s2) {
  float s = sqrtf(s2);
  if (s <= 0.8f) {
    float g = 0.0f;
#pragma unroll
    for (int k = 30; k >= 0; --k) g = fmaf(g, s2, 6.0f / (float)((2 * k + 3) * (2 * k + 5)));
    return s2 * s2 * s * g;
  }
  if (rho2 <= 0.0f) return 1.0f;
  float rho = sqrtf(rho2);
  return (1.0f + 2.0f * rho2) * s - 3.0f * rho2 * logf((1.0f + s) / rho);
}

__device__ inline double kstat_unit_d(double rho2, double s2) {
  double s = sqrt(s2);
  if (s <= 0.5) {
    double g = 0.0;
#pragma unroll
    for (int k = 26; k >= 0; --k) g = fma(g, s2, 6.0 / (double)((2 * k + 3) * (2 * k + 5)));
    return s2 * s2 * s * g;
  }
  if (rho2 <= 0.0) return 1.0;
  double rho = sqrt(rho2);
  return (1.0 + 2.0 * rho2) * s - 3.0 * rho2 * log((1.0 + s) / rho);
}

// atanh(s) - s = s^3 sum_{k>=0} s^(2k) / (2k+3); used for
// d k~/d r_s = (6 C / r_s) rho^2 (atanh(s) - s), from differentiating Eq. eq:kstat.
__device__ inline float atanh_minus_s_f(float rho2, float s2) {
  float s = sqrtf(s2);
  if (s <= 0.5f) {
    float g = 0.0f;
#pragma unroll
    for (int k = 12; k >= 0; --k) g = fmaf(g, s2, 1.0f / (float)(2 * k + 3));
    return s2 * s * g;
  }
  if (rho2 <= 0.0f) return 0.0f;  // multiplied by rho^2 = 0 by the caller
  return logf((1.0f + s) / sqrtf(rho2)) - s;
}

__device__ inline double atanh_minus_s_d(double rho2, double s2) {
  double s = sqrt(s2);
  if (s <= 0.3) {
    double g = 0.0;
#pragma unroll
    for (int k = 18; k >= 0; --k) g = fma(g, s2, 1.0 / (double)(2 * k + 3));
    return s2 * s * g;
  }
  if (rho2 <= 0.0) return 0.0;
  return log((1.0 + s) / sqrt(rho2)) - s;
}

// ---------------------------------------------------------------- error-free FP64
// Knuth's TwoSum and the FMA form of Dekker's TwoProduct: a + b = s + e and
// a * b = p + e exactly, with s = fl(a + b), p = fl(a * b).
__host__ __device__ inline void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double z = s - a;
  e = (a - (s - z)) + (b - z);
}
__host__ __device__ inline void two_prod(double a, double b, double& p, double& e) {
  p = a * b;
  e = fma(a, b, -p);
}

// 1 - |x - c|^2 / r^2 for FP64 points x, c (dim coordinates each) and
// radius^2 given exactly as r2h + r2l, with a relative error of a
// few units in the last place however close |x - c| is to r: each difference
// is split exactly into t + e (TwoSum), each square into p + pe
// (TwoProduct), the squared distance is carried as a double-double, and the
// cancelling subtraction r^2 - |x - c|^2 is done on the double-double pair.
__device__ inline double one_minus_ratio(const double* x, const double* c, int dim, double r2h, double r2l) {
  double hi = 0.0, lo = 0.0;
  for (int k = 0; k < dim; ++k) {
    double t, e, p, pe, s, se;
    two_sum(x[k], -c[k], t, e);
    two_prod(t, t, p, pe);
    two_sum(hi, p, s, se);
    hi = s;
    lo += se + pe + 2.0 * t * e;
  }
  double nh, nl;
  two_sum(r2h, -hi, nh, nl);
  nl += r2l - lo;
  return (nh + nl) / r2h * (1.0 - r2l / r2h);
}

// Sum of products a[m] b[m] over the set bits m of `bits`, compensated
// (TwoProduct + TwoSum, Ogita-Rump-Oishi Dot2): as accurate as if computed in
// twice the precision and rounded, so a sum that cancels keeps its digits.
__device__ inline double dot2_bits(const double* a, const double* b, uint32_t bits) {
  double s = 0.0, c = 0.0;
  while (bits) {
    const int m = __ffs(bits) - 1;
    bits &= bits - 1u;
    double p, pe, t, te;
    two_prod(a[m], b[m], p, pe);
    two_sum(s, p, t, te);
    s = t;
    c += te + pe;
  }
  return s + c;
}

// exp(-t) for t >= 0, the squared-exponential core exp(-d^2 / (2 l^2)) at
// t = d^2 / (2 l^2).  FP64: exp.  FP32 path: t split as th + tl (th its FP32
// rounding) and exp(-t) = expf(-th) (1 - tl), so the rounding of t to FP32
// (relative 2^-24, absolute 2^-24 t) does not enter the result.
template <typename T>
__device__ inline double sqexp_core(double t) {
  if (sizeof(T) == 8) return exp(-t);
  const float th = (float)t;
  const double tl = t - (double)th;
  return (double)expf(-th) * (1.0 - tl);
}

template <typename T> struct Real;
template <> struct Real<float> {
  __device__ static float kstat(float r2, float s2) { return kstat_unit_f(r2, s2); }
  __device__ static float dk(float r2, float s2) { return atanh_minus_s_f(r2, s2); }
};
template <> struct Real<double> {
  __device__ static double kstat(double r2, double s2) { return kstat_unit_d(r2, s2); }
  __device__ static double dk(double r2, double s2) { return atanh_minus_s_d(r2, s2); }
};

// The same error-free transformations in FP32: a + b = s + e, a * b = p + e.
__device__ inline void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}
__device__ inline void two_prod_f(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// |x_p - x_j|^2 as a double-float pair eh + el from coordinates given as
// double-float pairs (hi, lo): each difference exact (TwoSum on the high
// parts, plus the low parts), each square exact (TwoProduct, plus the cross
// and square terms of the correction), the sum carried as a pair.  The
// correction of a difference is as large as the rounding of the coordinates
// to FP32 (about 2^-24 |x|), so the high word alone is NOT d^2 to FP32
// accuracy: use eh + el.
__device__ inline void dist2_pair_f(const float2* __restrict__ xhl, int dim, int64_t p, int64_t j, float& eh,
                                    float& el) {
  eh = 0.f;
  el = 0.f;
  for (int k = 0; k < dim; ++k) {
    const float2 u = xhl[p * dim + k], w = xhl[j * dim + k];
    float t, e;
    two_sum_f(u.x, -w.x, t, e);
    e += u.y - w.y;
    float sq, sqe;
    two_prod_f(t, t, sq, sqe);
    sqe = fmaf(2.f * t, e, fmaf(e, e, sqe));
    float sum, se;
    two_sum_f(eh, sq, sum, se);
    eh = sum;
    el += se + sqe;
  }
}
// r^2 - (eh + el) for r^2 = rh + rl, on the pairs (no cancellation), rounded once.
__device__ inline float pair_gap_f(float rh, float rl, float eh, float el) {
  float nh, nl;
  two_sum_f(rh, -eh, nh, nl);
  nl += rl - el;
  return nh + nl;
}

// Compensated FP32 accumulation of products: the product's rounding error
// (FMA) and each addition's rounding error (Knuth's TwoSum) are carried in a
// second float, so a per-thread partial dot product keeps FP64-class accuracy
// without FP64 arithmetic; partials are then combined in FP64.
struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ inline void add(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float t = s + p;
    const float z = t - s;
    c += ((s - (t - z)) + (p - z)) + e;
    s = t;
  }
  __device__ inline double value() const { return (double)s + (double)c; }
};

// Sum partials part[b * stride + t] over blocks b < nblk for t < width with all
// threads of the block, in a fixed order; result in out[t] (shared).  Each
// thread keeps 16 predicated L2 loads in flight per round (no dependent tail).
__device__ inline void block_sum_partials(const double* part, int nblk, int width, int stride, double* out,
                                   double* scratch /* >= blockDim.x doubles */) {
  const int groups = blockDim.x / width;  // width <= 2 kMaxCols < blockDim.x
  const int t = threadIdx.x % width, grp = threadIdx.x / width;
  double a[4] = {0, 0, 0, 0};
  if (grp < groups) {
    for (int b0 = grp; b0 < nblk; b0 += 16 * groups) {
      double v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int b = b0 + u * groups;
        v[u] = b < nblk ? __ldcg(part + (int64_t)b * stride + t) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) a[u & 3] += v[u];
    }
  }
  scratch[threadIdx.x] = (a[0] + a[1]) + (a[2] + a[3]);
  __syncthreads();
  if (threadIdx.x < width) {
    double s = 0.0;
    for (int g2 = 0; g2 < groups; ++g2) s += scratch[g2 * width + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// alpha_c = rho_c / p_c^T q_c of iteration it for the columns still running
// (Saad, Alg. 6.18; rho = r^T M^-1 r, = |r|^2 without a preconditioner), with
// pq = p^T q per column already summed; threads c < kp of the calling block
// each finish one column.  A non-positive or non-finite p^T q is a breakdown.
__device__ inline void cg_alpha_finish(gp::CgState* st, int it, const double* pq, int k, int kp,
                                       double* hist_alpha, int m_hist) {
  if (threadIdx.x < kp) {
    const int c = threadIdx.x;
    double a = 0.0;
    if (c < k && !st->donep[it & 1][c]) {
      const double d = pq[c];
      if (!(d > 0.0) || !isfinite(d)) {
        st->status = GP_ERR_NOT_SPD;
        st->bad_col = c;
      } else {
        a = st->rrp[it & 1][c] / d;
        if (it < m_hist) {
          hist_alpha[it * gp::kMaxCols + c] = a;
          st->steps[c] = it + 1;
        }
      }
    }
    st->alpha[c] = a;
  }
}

__device__ inline unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace gpd

#define GP_CHECK(call)                        \
  do {                                        \
    int _s = (call);                          \
    if (_s != GP_OK) return _s;               \
  } while (0)

#define GP_CUDA(call)                                   \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return gp::cuda_status(_e);  \
  } while (0)

#define GP_LAUNCH_CHECK() GP_CUDA(cudaGetLastError())
