// C ABI of libgpsparse (see include/gpsparse.h): argument checks, host/device
// staging, buffer management and the order of the pipeline stages.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <thread>
#include <vector>

#include "gp_internal.cuh"

namespace gp {

int cuda_status(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return GP_ERR_OOM;
  }
  return GP_ERR_CUDA;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int ensure(gp_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return GP_OK;
  if (c->flags & GP_FLAG_FAULT_OOM) return GP_ERR_OOM;  // injected (tests of the error path)
  if (b.p) {
    GP_CUDA(cudaStreamSynchronize(c->stream));
    GP_CUDA(cudaFree(b.p));
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = bytes + bytes / 8 + 256;
  GP_CUDA(cudaMalloc(&b.p, want));
  b.cap = want;
  return GP_OK;
}

int ensure_pinned(gp_ctx* c, size_t bytes) {
  if (c->pinned_cap >= bytes) return GP_OK;
  if (c->pinned) {
    GP_CUDA(cudaStreamSynchronize(c->stream));
    GP_CUDA(cudaFreeHost(c->pinned));
    c->pinned = nullptr;
    c->pinned_cap = 0;
  }
  size_t want = bytes < 4096 ? 4096 : bytes;
  GP_CUDA(cudaMallocHost(&c->pinned, want));
  c->pinned_cap = want;
  return GP_OK;
}

int kernel_events(gp_ctx* c) {
  if (c->kev_ready) return GP_OK;
  for (int i = 0; i < (int)(sizeof(c->kev) / sizeof(c->kev[0])); ++i) GP_CUDA(cudaEventCreate(&c->kev[i]));
  c->kev_ready = true;
  return GP_OK;
}

double event_ms(cudaEvent_t a, cudaEvent_t b) {
  float t = 0.f;
  if (cudaEventElapsedTime(&t, a, b) != cudaSuccess) {
    cudaGetLastError();
    return 0.0;
  }
  return t;
}

}  // namespace gp

namespace {

// gp_lml_grad_batched, grouped CG launches: instances per wave (one worker
// context each)
constexpr int kBatchWave = 256;

void reset_counters(gp_ctx* c, int flags) {
  c->flags = flags;
  c->launches = 0;
  c->t_spmm = c->t_fill = c->t_adj = 0.0;
  c->n_spmm = 0;
  c->bad_col = -1;
  c->spmm_variant = -1;
}

void fill_counters(const gp_ctx* c, gp_info* info) {
  info->launches = c->launches;
  info->status_detail = c->bad_col;
  info->n_spmm = c->n_spmm;
  info->t_spmm_kernel_ms = c->t_spmm;
  info->t_fill_kernel_ms = c->t_fill;
  info->t_adjoint_kernel_ms = c->t_adj;
  info->spmm_variant = c->spmm_variant;
}

int check_desc(const gp_kernel_desc* d) {
  if (!d) return GP_ERR_INVALID_ARG;
  if (d->dim < 1 || d->n_funcs < 1 || d->n_bumps < 1 || !(d->beta > 0.0) || !isfinite(d->beta))
    return GP_ERR_INVALID_ARG;
  if (d->core != GP_CORE_NONE && d->core != GP_CORE_SQEXP) return GP_ERR_INVALID_ARG;
  if (d->dim > gp::kMaxDim || d->n_funcs > gp::kMaxFuncs || (int64_t)d->n_funcs * d->n_bumps > gp::kMaxBumps)
    return GP_ERR_UNSUPPORTED;
  return GP_OK;
}

int check_h(const gp_ctx* c, const double* h) {
  if (!h) return GP_ERR_INVALID_ARG;
  const int np = c->dim + 2;
  for (int b = 0; b < c->nb; ++b) {
    for (int t = 0; t < np; ++t)
      if (!isfinite(h[b * np + t])) return GP_ERR_INVALID_ARG;
    if (!(h[b * np + c->dim] > 0.0)) return GP_ERR_INVALID_ARG;  // radius
  }
  const double rs = h[c->nb * np], A = h[c->nb * np + 1], s2 = h[c->nb * np + 2];
  if (!isfinite(rs) || !isfinite(A) || !isfinite(s2)) return GP_ERR_INVALID_ARG;
  if (!(rs > 0.0) || !(A >= 0.0) || !(s2 > 0.0)) return GP_ERR_INVALID_ARG;
  if (c->core == GP_CORE_SQEXP) {
    const double l = h[c->nb * np + 3];
    if (!isfinite(l) || !(l > 0.0)) return GP_ERR_INVALID_ARG;
  }
  return GP_OK;
}

int check_opts(const gp_opts* o, bool need_probes) {
  if (!o) return GP_ERR_INVALID_ARG;
  if (o->precision != GP_FP64 && o->precision != GP_FP32_MIXED) return GP_ERR_INVALID_ARG;
  if (o->max_iter < 1 || !(o->cg_rtol > 0.0) || !isfinite(o->cg_rtol)) return GP_ERR_INVALID_ARG;
  if (o->precond_block != 0 && o->precond_block != 8 && o->precond_block != 16 && o->precond_block != 32 &&
      o->precond_block != 64 && o->precond_block != 128)
    return GP_ERR_INVALID_ARG;
  if (o->batch_workers < 0 || o->batch_workers > 16) return GP_ERR_INVALID_ARG;
  if (need_probes) {
    if (o->n_probes < 1 || o->n_probes > gp::kMaxProbes) return GP_ERR_INVALID_ARG;
    // SLQ keeps lanczos_steps coefficients per column; the Taylor series keeps none
    const int max_steps = (o->flags & GP_FLAG_LOGDET_TAYLOR) ? 4096 : gp::kMaxLanczos;
    if (o->lanczos_steps < 1 || o->lanczos_steps > max_steps) return GP_ERR_INVALID_ARG;
  }
  return GP_OK;
}

// Make a device-resident copy of a caller array if it lives on the host.
int stage_in(gp_ctx* c, gp::DevBuf& buf, const double* src, size_t count, const double** out) {
  if (count == 0) {
    *out = src;
    return GP_OK;
  }
  if (gp::is_device_ptr(src)) {
    *out = src;
    return GP_OK;
  }
  GP_CHECK(gp::ensure(c, buf, count * sizeof(double)));
  GP_CUDA(cudaMemcpyAsync(buf.p, src, count * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  *out = (const double*)buf.p;
  return GP_OK;
}

int copy_out(gp_ctx* c, void* dst, const void* src_dev, size_t bytes) {
  if (bytes == 0) return GP_OK;
  GP_CUDA(cudaMemcpyAsync(dst, src_dev, bytes, gp::is_device_ptr(dst) ? cudaMemcpyDeviceToDevice
                                                                       : cudaMemcpyDeviceToHost,
                          c->stream));
  return GP_OK;
}

struct Timer {
  gp_ctx* c;
  explicit Timer(gp_ctx* cc) : c(cc) {}
  void mark(int i) { cudaEventRecord(c->ev[i], c->stream); }
  double ms(int a, int b) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->ev[a], c->ev[b]) != cudaSuccess) {
      cudaGetLastError();
      return 0.0;
    }
    return t;
  }
};

int read_scalars(gp_ctx* c, gp::AsmScalars* hs) {
  GP_CHECK(gp::ensure_pinned(c, sizeof(gp::AsmScalars)));
  GP_CUDA(cudaMemcpyAsync(c->pinned, c->asm_s.p, sizeof(gp::AsmScalars), cudaMemcpyDeviceToHost, c->stream));
  GP_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(hs, c->pinned, sizeof(gp::AsmScalars));
  return GP_OK;
}

// One evaluation between its phases: the batched path runs the CG runs of
// many instances together between the front and the back of each.
struct EvalRun {
  const double *xd = nullptr, *yd = nullptr;
  int64_t n = 0;
  int nv = 0, k = 0, kp = 0;
  bool taylor = false;
  int iters = 0, lanczos_iters = 0;
  double max_rel = 0.0;
  int cg_status = GP_OK;
};

// Stage the inputs in, assemble, and set up the preconditioner and the terms
// of the inactive points.
int eval_front(gp_ctx* c, const double* x, const double* y, int64_t n, const double* h, const gp_opts* o,
               EvalRun* r) {
  if (!c || n < 0 || (n > 0 && (!x || !y))) return GP_ERR_INVALID_ARG;
  GP_CHECK(check_h(c, h));
  GP_CHECK(check_opts(o, true));
  GP_CUDA(cudaSetDevice(c->device));
  reset_counters(c, o->flags);
  Timer tm(c);
  tm.mark(0);
  r->n = n;
  GP_CHECK(stage_in(c, c->x_in, x, (size_t)n * c->dim, &r->xd));
  GP_CHECK(stage_in(c, c->y_in, y, (size_t)n, &r->yd));
  GP_CHECK(gp::assemble(c, r->xd, n, h, o->precision));
  tm.mark(1);
  if (o->flags & (GP_FLAG_FAULT_NOT_SPD | GP_FLAG_FAULT_NAN)) GP_CHECK(gp::inject_matrix_fault(c, o->flags));
  GP_CHECK(gp::precond_setup(c, o->precond_block));
  GP_CHECK(gp::inactive_terms(c, r->yd));
  r->nv = o->n_probes;
  r->k = 1 + r->nv;
  r->kp = (r->k + 3) / 4 * 4;
  // the log-determinant estimator: SLQ, or the truncated Taylor series the
  // paper cites (FP32 path; lanczos_steps terms on the same probes)
  r->taylor = (o->flags & GP_FLAG_LOGDET_TAYLOR) != 0;
  if (r->taylor && o->precision != GP_FP32_MIXED) return GP_ERR_UNSUPPORTED;
  return GP_OK;
}

// The solves of one evaluation on its own context.
int eval_solve(gp_ctx* c, const gp_opts* o, EvalRun* r) {
  const int nv = r->nv, k = r->k, kp = r->kp;
  const double* yd = r->yd;
  if (o->precision == GP_FP64) {
    r->cg_status = gp::cg_run_fp64(c, k, yd, nv, o->seed, o->lanczos_steps, o->max_iter, o->cg_rtol,
                                   o->check_every, &r->iters, &r->max_rel);
  } else if (r->taylor) {
    // the solves alone (preconditioned when asked), then the series on V = C^k Z
    r->cg_status = gp::cg_run(c, k, kp, yd, nv, o->seed, 0, o->max_iter, o->cg_rtol, o->check_every, &r->iters,
                              &r->max_rel, c->pc_block > 0);
    if (r->cg_status == GP_OK || r->cg_status == GP_ERR_NOT_CONVERGED)
      GP_CHECK(gp::taylor_logdet(c, nv, kp, o->lanczos_steps));
  } else if (c->pc_block == 0) {
    // one plain CG run: its first lanczos_steps coefficients feed SLQ
    r->cg_status = gp::cg_run(c, k, kp, yd, nv, o->seed, o->lanczos_steps, o->max_iter, o->cg_rtol,
                              o->check_every, &r->iters, &r->max_rel, false);
  } else {
    // SLQ needs the Lanczos coefficients of Khat itself from the probes: a
    // short plain run of lanczos_steps iterations (expected not to converge),
    // reduced to SLQ terms before the preconditioned run reuses the CG state
    double lanczos_rel = 0.0;
    // (one check interval of lanczos_steps iterations: the run always goes to
    // its cap, so shorter intervals only add host checks and idle launches)
    const int lst = gp::cg_run(c, k, kp, yd, nv, o->seed, o->lanczos_steps, o->lanczos_steps, o->cg_rtol,
                               o->lanczos_steps, &r->lanczos_iters, &lanczos_rel, false);
    if (lst != GP_OK && lst != GP_ERR_NOT_CONVERGED) return lst;
    // the eigen-solves overlap the preconditioned run (side stream)
    GP_CHECK(gp::slq(c, nv, kp, true));
    // the preconditioned solves start from the Lanczos run's iterate
    r->cg_status = gp::cg_run(c, k, kp, yd, nv, o->seed, 0, o->max_iter, o->cg_rtol, o->check_every, &r->iters,
                              &r->max_rel, true, true);
    const int jst = gp::slq_join(c);
    if (jst != GP_OK) return jst;
  }
  return GP_OK;
}

// Everything after the solves: the quadratic form, SLQ when no
// preconditioned run overlapped it, the adjoint gradient, and ln L.
int eval_back(gp_ctx* c, const gp_opts* o, const EvalRun& r, double* lml, double* grad, gp_info* info) {
  const int64_t n = r.n;
  const int nv = r.nv, k = r.k, kp = r.kp;
  const double* yd = r.yd;
  const bool taylor = r.taylor;
  const int cg_status = r.cg_status, iters = r.iters, lanczos_iters = r.lanczos_iters;
  const double max_rel = r.max_rel;
  Timer tm(c);
  if (cg_status != GP_OK && cg_status != GP_ERR_NOT_CONVERGED) return cg_status;
  GP_CHECK(gp::quad_form(c, yd, kp));
  if (!taylor && (o->precision == GP_FP64 || c->pc_block == 0)) GP_CHECK(gp::slq(c, nv, kp));
  tm.mark(2);
  if (grad) GP_CHECK(gp::adjoint(c, nv, kp));
  tm.mark(3);
  gp::AsmScalars hs;
  GP_CHECK(read_scalars(c, &hs));
  if (!isfinite(hs.inact_y2)) return GP_ERR_INVALID_ARG;  // a non-finite target outside every bump
  if (c->n_act > 0 && hs.status != GP_OK) return hs.status;
  if (c->pc_block > 0 && hs.pc_status != GP_OK) return hs.pc_status;
  const double s2 = c->sigma2;
  const double n_in = (double)(n - c->n_act);
  const double logdet = hs.sum_log_d * (c->n_act > 0) + hs.slq_mean + n_in * log(s2);
  const double quad = hs.quad_form + hs.inact_y2 / s2;
  *lml = -0.5 * quad - 0.5 * logdet;
  if (grad) {
    const int np = c->dim + 2;
    const size_t nbp = (size_t)c->nb * np;
    std::vector<double> gb(nbp, 0.0);
    if (c->n_act > 0) {
      GP_CHECK(gp::ensure_pinned(c, nbp * sizeof(double)));
      GP_CUDA(cudaMemcpyAsync(c->pinned, c->grad_bump.p, nbp * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      GP_CUDA(cudaStreamSynchronize(c->stream));
      memcpy(gb.data(), c->pinned, nbp * sizeof(double));
    }
    const bool core = c->core == GP_CORE_SQEXP;
    std::vector<double> out(nbp + 3 + (core ? 1 : 0));
    for (size_t q = 0; q < nbp; ++q) out[q] = gb[q];
    const bool act = c->n_act > 0;
    out[nbp] = act ? hs.grad_rs : 0.0;
    out[nbp + 1] = act ? hs.grad_A : 0.0;
    out[nbp + 2] = (act ? hs.grad_s2 : 0.0) + 0.5 * hs.inact_y2 / (s2 * s2) - 0.5 * n_in / s2;
    if (core) out[nbp + 3] = act ? hs.grad_l : 0.0;
    if (gp::is_device_ptr(grad)) {
      GP_CHECK(gp::ensure_pinned(c, out.size() * sizeof(double)));
      memcpy(c->pinned, out.data(), out.size() * sizeof(double));
      GP_CUDA(cudaMemcpyAsync(grad, c->pinned, out.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      GP_CUDA(cudaStreamSynchronize(c->stream));
    } else {
      memcpy(grad, out.data(), out.size() * sizeof(double));
    }
  }
  if (info) {
    info->n = n;
    info->n_active = c->n_act;
    info->nnz = c->nnz;
    info->iters = iters;
    info->status_detail = -1;
    info->max_rel_resid = max_rel;
    info->quad_form = quad;
    info->logdet = logdet;
    info->logdet_stderr = nv > 1 ? sqrt(hs.slq_var / nv) : 0.0;
    info->t_assemble_ms = tm.ms(0, 1);
    info->t_solve_ms = tm.ms(1, 2);
    info->t_grad_ms = grad ? tm.ms(2, 3) : 0.0;
    info->cell_size = c->grid.h;
    info->n_cells = c->grid.ncells;
    info->kp = o->precision == GP_FP64 ? k : kp;
    info->lanczos_iters = lanczos_iters;
    info->precond_block = c->pc_block;
    fill_counters(c, info);
  }
  return cg_status;
}

// Assemble, solve [y, probes], SLQ, optional adjoint.
int evaluate(gp_ctx* c, const double* x, const double* y, int64_t n, const double* h, const gp_opts* o,
             double* lml, double* grad, gp_info* info) {
  if (!c || !lml) return GP_ERR_INVALID_ARG;
  EvalRun r;
  GP_CHECK(eval_front(c, x, y, n, h, o, &r));
  GP_CHECK(eval_solve(c, o, &r));
  return eval_back(c, o, r, lml, grad, info);
}

}  // namespace

extern "C" {

int64_t gp_n_params(const gp_kernel_desc* d) {
  if (!d) return -1;
  return (int64_t)d->n_funcs * d->n_bumps * (d->dim + 2) + 3 + (d->core == GP_CORE_SQEXP ? 1 : 0);
}

int gp_sparsity_estimate(const gp_kernel_desc* d, const double* h, double domain_volume, double* s, double* grad) {
  GP_CHECK(check_desc(d));
  if (!h || !s || !(domain_volume > 0.0) || !isfinite(domain_volume)) return GP_ERR_INVALID_ARG;
  const int dim = d->dim, n1 = d->n_funcs, n2 = d->n_bumps, np = dim + 2;
  // Vol(dim, r) = pi^(dim/2) / Gamma(dim/2 + 1) r^dim
  const double unit = pow(M_PI, 0.5 * dim) / tgamma(0.5 * dim + 1.0);
  const double inv_v2 = 1.0 / (domain_volume * domain_volume);
  for (int b = 0; b < n1 * n2; ++b) {
    const double r = h[b * np + dim];
    if (!(r > 0.0) || !isfinite(r)) return GP_ERR_INVALID_ARG;
  }
  if (grad)
    for (int64_t q = 0; q < gp_n_params(d); ++q) grad[q] = 0.0;
  double total = 0.0;
  for (int i = 0; i < n1; ++i) {
    double vsum = 0.0;  // sum over the bumps of f_i of their ball volumes
    for (int j = 0; j < n2; ++j) vsum += unit * pow(h[(i * n2 + j) * np + dim], dim);
    total += vsum * vsum;  // = sum_j sum_k Vol(r_ij) Vol(r_ik)
    if (grad)
      for (int j = 0; j < n2; ++j) {
        const double r = h[(i * n2 + j) * np + dim];
        grad[(i * n2 + j) * np + dim] = 2.0 * vsum * dim * unit * pow(r, dim) / r * inv_v2;
      }
  }
  *s = total * inv_v2;
  return GP_OK;
}

int gp_augmented(const gp_kernel_desc* d, const double* h, double domain_volume, double lml, const double* lml_grad,
                 double* value, double* grad, double* s_out) {
  if (!value || (grad && !lml_grad) || !isfinite(lml)) return GP_ERR_INVALID_ARG;
  GP_CHECK(check_desc(d));
  const int64_t np = gp_n_params(d);
  std::vector<double> ds(grad ? (size_t)np : 0);
  double s = 0.0;
  GP_CHECK(gp_sparsity_estimate(d, h, domain_volume, &s, grad ? ds.data() : nullptr));
  *value = (2.0 - s) * lml;
  if (grad)
    for (int64_t q = 0; q < np; ++q) grad[q] = (2.0 - s) * lml_grad[q] - lml * ds[q];
  if (s_out) *s_out = s;
  return GP_OK;
}

void gp_default_opts(gp_opts* o) {
  if (!o) return;
  o->precision = GP_FP32_MIXED;
  o->n_probes = 32;
  o->lanczos_steps = 50;
  o->max_iter = 10000;
  o->cg_rtol = 1e-6;
  o->seed = 0x5eedull;
  o->check_every = 16;
  o->flags = 0;
  o->precond_block = 128;
  o->batch_workers = 0;
}

int gp_create(gp_ctx** out, const gp_kernel_desc* desc, int device, void* stream) {
  if (!out) return GP_ERR_INVALID_ARG;
  *out = nullptr;
  GP_CHECK(check_desc(desc));
  GP_CUDA(cudaSetDevice(device));
  gp_ctx* c = new (std::nothrow) gp_ctx();
  if (!c) return GP_ERR_OOM;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  c->dim = desc->dim;
  c->n1 = desc->n_funcs;
  c->n2 = desc->n_bumps;
  c->nb = desc->n_funcs * desc->n_bumps;
  c->beta = desc->beta;
  c->core = desc->core;
  int st = GP_OK;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) st = GP_ERR_CUDA;
  if (st == GP_OK) c->num_sms = prop.multiProcessorCount;
  if (st == GP_OK) st = gp::ensure(c, c->cg, sizeof(gp::CgState));
  if (st == GP_OK) st = gp::ensure(c, c->asm_s, sizeof(gp::AsmScalars));
  if (st == GP_OK && cudaMemsetAsync(c->cg.p, 0, sizeof(gp::CgState), c->stream) != cudaSuccess) st = GP_ERR_CUDA;
  if (st == GP_OK && cudaMemsetAsync(c->asm_s.p, 0, sizeof(gp::AsmScalars), c->stream) != cudaSuccess)
    st = GP_ERR_CUDA;
  for (int i = 0; i < 8 && st == GP_OK; ++i)
    if (cudaEventCreate(&c->ev[i]) != cudaSuccess) st = GP_ERR_CUDA;
  if (st == GP_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = GP_ERR_CUDA;
  if (st != GP_OK) {
    gp_destroy(c);
    return st;
  }
  *out = c;
  return GP_OK;
}

int gp_destroy(gp_ctx* c) {
  if (!c) return GP_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->aux_stream) cudaStreamSynchronize(c->aux_stream);
  gp::DevBuf* bufs[] = {&c->x_in,   &c->y_in,   &c->out_tmp,    &c->bump,      &c->mask0,     &c->F0,
                        &c->pos,    &c->keys,   &c->vals,       &c->keys2,     &c->vals2,     &c->hist,
                        &c->hist_scan, &c->scan_part, &c->cells, &c->perm,     &c->skey,      &c->cellc,
                        &c->xr,     &c->xs,     &c->xhl, &c->Fs,  &c->Fhl,  &c->smask,     &c->dinv,      &c->dinv64,
                        &c->cnt,    &c->row_ptr, &c->col,       &c->val,       &c->X,         &c->R,
                        &c->P,      &c->Q,      &c->zbits,      &c->part_a,    &c->part_b,    &c->part_c,
                        &c->hist_alpha, &c->hist_beta, &c->g,   &c->grad_part, &c->grad_bump, &c->cg,
                        &c->asm_s,  &c->csr_tmp, &c->bcnt,     &c->brp,       &c->bcol,      &c->bmask,
                        &c->bval,   &c->slq_g,  &c->pc_Minv,    &c->pc_part,   &c->Z,
                        &c->xstar_in, &c->pred_tmp, &c->slq_steps, &c->taylor,
                        &c->w_cnt,  &c->w_tseg, &c->w_trun,     &c->w_trec,    &c->w_segd,    &c->w_runs,
                        &c->w_rec,  &c->pv_B,   &c->pv_prior, &c->grp_inst, &c->grp_map};
  for (gp::DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (c->pinned) cudaFreeHost(c->pinned);
  for (int i = 0; i < 8; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  if (c->kev_ready)
    for (cudaEvent_t e : c->kev) cudaEventDestroy(e);
  for (auto& gr : c->cg_graph)
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  for (cudaEvent_t e : c->aux_ev)
    if (e) cudaEventDestroy(e);
  for (gp_ctx* w : c->workers) gp_destroy(w);
  if (c->owned_stream) cudaStreamDestroy(c->owned_stream);
  delete c;
  return GP_OK;
}

int gp_set_stream(gp_ctx* c, void* stream) {
  if (!c) return GP_ERR_INVALID_ARG;
  GP_CUDA(cudaSetDevice(c->device));
  GP_CUDA(cudaStreamSynchronize(c->stream));
  c->stream = (cudaStream_t)stream;
  return GP_OK;
}

int gp_assemble(gp_ctx* c, const double* x, int64_t n, const double* h, const gp_opts* o, gp_info* info) {
  if (!c || n < 0 || (n > 0 && !x) || !o) return GP_ERR_INVALID_ARG;
  if (o->precision != GP_FP64 && o->precision != GP_FP32_MIXED) return GP_ERR_INVALID_ARG;
  GP_CHECK(check_h(c, h));
  GP_CUDA(cudaSetDevice(c->device));
  reset_counters(c, o->flags);
  Timer tm(c);
  tm.mark(0);
  const double* xd = nullptr;
  GP_CHECK(stage_in(c, c->x_in, x, (size_t)n * c->dim, &xd));
  GP_CHECK(gp::assemble(c, xd, n, h, o->precision));
  tm.mark(1);
  GP_CUDA(cudaStreamSynchronize(c->stream));
  if (info) {
    memset(info, 0, sizeof(*info));
    info->n = n;
    info->n_active = c->n_act;
    info->nnz = c->nnz;
    info->status_detail = -1;
    info->t_assemble_ms = tm.ms(0, 1);
    info->cell_size = c->grid.h;
    info->n_cells = c->grid.ncells;
    fill_counters(c, info);
  }
  return GP_OK;
}

int gp_get_csr(gp_ctx* c, int64_t* row_ptr, int32_t* col, double* val, int32_t* perm, int64_t sizes[2]) {
  if (!c || !sizes) return GP_ERR_INVALID_ARG;
  if (!c->assembled) return GP_ERR_NOT_ASSEMBLED;
  GP_CUDA(cudaSetDevice(c->device));
  sizes[0] = c->n_act;
  sizes[1] = c->nnz;
  if (c->n_act == 0) {
    if (row_ptr) {
      int64_t z = 0;
      if (gp::is_device_ptr(row_ptr)) GP_CUDA(cudaMemcpy(row_ptr, &z, sizeof(z), cudaMemcpyHostToDevice));
      else *row_ptr = 0;
    }
    return GP_OK;
  }
  if (row_ptr) GP_CHECK(copy_out(c, row_ptr, c->row_ptr.p, (size_t)(c->n_act + 1) * sizeof(int64_t)));
  if (col) GP_CHECK(copy_out(c, col, c->col.p, (size_t)c->nnz * sizeof(int32_t)));
  if (perm) GP_CHECK(copy_out(c, perm, c->vals.p, (size_t)c->n_act * sizeof(int32_t)));
  if (val) {
    GP_CHECK(gp::ensure(c, c->csr_tmp, (size_t)c->nnz * sizeof(double)));
    GP_CHECK(gp::csr_unscaled(c, (double*)c->csr_tmp.p));
    GP_CHECK(copy_out(c, val, c->csr_tmp.p, (size_t)c->nnz * sizeof(double)));
  }
  GP_CUDA(cudaStreamSynchronize(c->stream));
  return GP_OK;
}

namespace {

// alpha = K^-1 y (original point order) into the device array out (c->n
// doubles) with the last assembled K: CG on the Jacobi-scaled active block
// (block-Jacobi preconditioned in FP32 when opts ask for it), y_i / sigma^2
// on the rows outside every bump.
int solve_alpha(gp_ctx* c, const double* yd, const gp_opts* o, double* out, int* iters, double* max_rel) {
  GP_CHECK(gp::precond_setup(c, o->precond_block));
  int st;
  if (c->precision == GP_FP64)
    st = gp::cg_run_fp64(c, 1, yd, 0, o->seed, 0, o->max_iter, o->cg_rtol, o->check_every, iters, max_rel);
  else
    st = gp::cg_run(c, 1, 4, yd, 0, o->seed, 0, o->max_iter, o->cg_rtol, o->check_every, iters, max_rel, true);
  if (st != GP_OK && st != GP_ERR_NOT_CONVERGED) return st;
  if (c->n > 0) GP_CHECK(gp::alpha_out(c, yd, out, 4));
  return st;
}

void solve_info(const gp_ctx* c, int iters, double max_rel, double ms, gp_info* info) {
  memset(info, 0, sizeof(*info));
  info->n = c->n;
  info->n_active = c->n_act;
  info->nnz = c->nnz;
  info->iters = iters;
  info->status_detail = -1;
  info->max_rel_resid = max_rel;
  info->t_solve_ms = ms;
  info->cell_size = c->grid.h;
  info->n_cells = c->grid.ncells;
  info->kp = 4;
  info->precond_block = c->pc_block;
  fill_counters(c, info);
}

}  // namespace

int gp_solve(gp_ctx* c, const double* y, double* alpha, const gp_opts* o, gp_info* info) {
  if (!c || !alpha || !o) return GP_ERR_INVALID_ARG;
  if (!c->assembled) return GP_ERR_NOT_ASSEMBLED;
  GP_CHECK(check_opts(o, false));
  if (c->n > 0 && !y) return GP_ERR_INVALID_ARG;
  GP_CUDA(cudaSetDevice(c->device));
  reset_counters(c, o->flags);
  Timer tm(c);
  tm.mark(0);
  const double* yd = nullptr;
  GP_CHECK(stage_in(c, c->y_in, y, (size_t)c->n, &yd));
  double* out = alpha;
  const bool dev = gp::is_device_ptr(alpha);
  if (!dev) {
    GP_CHECK(gp::ensure(c, c->out_tmp, (size_t)c->n * sizeof(double)));
    out = (double*)c->out_tmp.p;
  }
  int iters = 0;
  double max_rel = 0.0;
  const int st = solve_alpha(c, yd, o, out, &iters, &max_rel);
  if (st != GP_OK && st != GP_ERR_NOT_CONVERGED) return st;
  if (!dev && c->n > 0)
    GP_CUDA(cudaMemcpyAsync(alpha, out, (size_t)c->n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  tm.mark(1);
  GP_CUDA(cudaStreamSynchronize(c->stream));
  if (info) solve_info(c, iters, max_rel, tm.ms(0, 1), info);
  return st;
}

int gp_predict(gp_ctx* c, const double* y, const double* xstar, int64_t n_star, double* mean, const gp_opts* o,
               gp_info* info) {
  if (!c || !o || n_star < 0 || (n_star > 0 && (!xstar || !mean))) return GP_ERR_INVALID_ARG;
  if (!c->assembled) return GP_ERR_NOT_ASSEMBLED;
  GP_CHECK(check_opts(o, false));
  if (c->n > 0 && !y) return GP_ERR_INVALID_ARG;
  GP_CUDA(cudaSetDevice(c->device));
  reset_counters(c, o->flags);
  Timer tm(c);
  tm.mark(0);
  const double *yd = nullptr, *xsd = nullptr;
  GP_CHECK(stage_in(c, c->y_in, y, (size_t)c->n, &yd));
  GP_CHECK(stage_in(c, c->xstar_in, xstar, (size_t)n_star * c->dim, &xsd));
  GP_CHECK(gp::ensure(c, c->out_tmp, (size_t)(c->n > 0 ? c->n : 1) * sizeof(double)));
  int iters = 0;
  double max_rel = 0.0;
  const int st = solve_alpha(c, yd, o, (double*)c->out_tmp.p, &iters, &max_rel);
  if (st != GP_OK && st != GP_ERR_NOT_CONVERGED) return st;
  double* md = mean;
  const bool dev = n_star > 0 && gp::is_device_ptr(mean);
  if (!dev && n_star > 0) {
    GP_CHECK(gp::ensure(c, c->pred_tmp, (size_t)n_star * sizeof(double)));
    md = (double*)c->pred_tmp.p;
  }
  GP_CHECK(gp::predict_mean(c, xsd, n_star, (const double*)c->out_tmp.p, md));
  if (!dev && n_star > 0)
    GP_CUDA(cudaMemcpyAsync(mean, md, (size_t)n_star * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  tm.mark(1);
  GP_CUDA(cudaStreamSynchronize(c->stream));
  if (info) solve_info(c, iters, max_rel, tm.ms(0, 1), info);
  return st;
}

int gp_predict_var(gp_ctx* c, const double* xstar, int64_t n_star, double* var, const gp_opts* o,
                   gp_info* info) {
  if (!c || !o || n_star < 0 || (n_star > 0 && (!xstar || !var))) return GP_ERR_INVALID_ARG;
  if (!c->assembled) return GP_ERR_NOT_ASSEMBLED;
  GP_CHECK(check_opts(o, false));
  GP_CUDA(cudaSetDevice(c->device));
  reset_counters(c, o->flags);
  Timer tm(c);
  tm.mark(0);
  const double* xsd = nullptr;
  GP_CHECK(stage_in(c, c->xstar_in, xstar, (size_t)n_star * c->dim, &xsd));
  double* vd = var;
  const bool dev = n_star > 0 && gp::is_device_ptr(var);
  if (!dev && n_star > 0) {
    GP_CHECK(gp::ensure(c, c->pred_tmp, (size_t)n_star * sizeof(double)));
    vd = (double*)c->pred_tmp.p;
  }
  int iters = 0;
  double max_rel = 0.0;
  const int st = gp::predict_var(c, xsd, n_star, vd, o, &iters, &max_rel);
  if (st != GP_OK && st != GP_ERR_NOT_CONVERGED) return st;
  if (!dev && n_star > 0)
    GP_CUDA(cudaMemcpyAsync(var, vd, (size_t)n_star * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  tm.mark(1);
  GP_CUDA(cudaStreamSynchronize(c->stream));
  if (info) solve_info(c, iters, max_rel, tm.ms(0, 1), info);
  return st;
}

int gp_lml(gp_ctx* c, const double* x, const double* y, int64_t n, const double* h, const gp_opts* o, double* lml,
           gp_info* info) {
  return evaluate(c, x, y, n, h, o, lml, nullptr, info);
}

int gp_lml_grad(gp_ctx* c, const double* x, const double* y, int64_t n, const double* h, const gp_opts* o,
                double* lml, double* grad, gp_info* info) {
  if (!grad) return GP_ERR_INVALID_ARG;
  return evaluate(c, x, y, n, h, o, lml, grad, info);
}

int gp_train(gp_ctx* c, const double* x, const double* y, int64_t n, double* h, const gp_opts* o,
             const gp_train_opts* t, double* trace, gp_info* info) {
  if (!c || !h || !o || !t) return GP_ERR_INVALID_ARG;
  if (t->objective < GP_OBJ_LML || t->objective > GP_OBJ_CONSTRAINED || t->n_steps < 0 || t->n_steps > 100000 ||
      !(t->lr > 0.0) || !isfinite(t->lr) || !(t->domain_volume > 0.0) || !isfinite(t->domain_volume) ||
      t->max_halvings < 0 || t->max_halvings > 1000)
    return GP_ERR_INVALID_ARG;
  double b1 = t->beta1, b2 = t->beta2, eps = t->eps;
  if (b1 == 0.0 && b2 == 0.0) {
    b1 = 0.9;
    b2 = 0.999;
  }
  if (eps == 0.0) eps = 1e-8;
  if (!(b1 >= 0.0 && b1 < 1.0) || !(b2 >= 0.0 && b2 < 1.0) || !(eps > 0.0) || !isfinite(eps))
    return GP_ERR_INVALID_ARG;
  const bool constrained = t->objective == GP_OBJ_CONSTRAINED;
  if (constrained && !(t->s_max > 0.0 && isfinite(t->s_max))) return GP_ERR_INVALID_ARG;
  const int halvings = t->max_halvings > 0 ? t->max_halvings : 30;
  GP_CHECK(check_h(c, h));
  const gp_kernel_desc d{c->dim, c->n1, c->n2, c->beta, c->core};
  const int64_t np = gp_n_params(&d);
  const int bp = c->dim + 2;
  // entries stepped in ln h: the bump radii, then r_s, A, sigma_n^2 (and l)
  std::vector<char> logp((size_t)np, 0);
  for (int b = 0; b < c->nb; ++b) logp[(size_t)b * bp + c->dim] = 1;
  for (int64_t q = (int64_t)c->nb * bp; q < np; ++q) logp[(size_t)q] = 1;
  if (!(h[(int64_t)c->nb * bp + 1] > 0.0)) return GP_ERR_INVALID_ARG;  // A
  std::vector<double> gl((size_t)np), ds((size_t)np), m((size_t)np, 0.0), v((size_t)np, 0.0), delta((size_t)np),
      hn((size_t)np);
  double s = 0.0;
  GP_CHECK(gp_sparsity_estimate(&d, h, t->domain_volume, &s, nullptr));
  if (constrained && !(s < t->s_max)) return GP_ERR_INVALID_ARG;
  for (int step = 0;; ++step) {
    double lml = 0.0;
    const int st = evaluate(c, x, y, n, h, o, &lml, gl.data(), info);
    if (st != GP_OK) return st;
    GP_CHECK(gp_sparsity_estimate(&d, h, t->domain_volume, &s, ds.data()));
    const bool aug = t->objective == GP_OBJ_AUGMENTED;
    const double obj = aug ? (2.0 - s) * lml : lml;
    if (trace) {
      trace[3 * step] = obj;
      trace[3 * step + 1] = lml;
      trace[3 * step + 2] = s;
    }
    if (step == t->n_steps) break;
    // Adam on theta (bias-corrected moments of d obj / d theta)
    const double c1 = 1.0 - pow(b1, step + 1), c2 = 1.0 - pow(b2, step + 1);
    for (int64_t q = 0; q < np; ++q) {
      const double gh = aug ? (2.0 - s) * gl[q] - lml * ds[q] : gl[q];  // d obj / d h_q
      const double g = logp[q] ? h[q] * gh : gh;
      if (!isfinite(g)) return GP_ERR_INVALID_ARG;
      m[q] = b1 * m[q] + (1.0 - b1) * g;
      v[q] = b2 * v[q] + (1.0 - b2) * g * g;
      delta[q] = t->lr * (m[q] / c1) / (sqrt(v[q] / c2) + eps);
    }
    // h_t = h(theta + f delta): f = 1, halved while the constraint fails
    double f = 1.0;
    for (int k = 0;; ++k) {
      for (int64_t q = 0; q < np; ++q) hn[q] = logp[q] ? h[q] * exp(f * delta[q]) : h[q] + f * delta[q];
      if (!constrained) break;
      double sn = 0.0;
      GP_CHECK(gp_sparsity_estimate(&d, hn.data(), t->domain_volume, &sn, nullptr));
      if (sn < t->s_max) break;
      if (k == halvings) {
        for (int64_t q = 0; q < np; ++q) hn[q] = h[q];  // no feasible step: stay
        break;
      }
      f *= 0.5;
    }
    memcpy(h, hn.data(), (size_t)np * sizeof(double));
  }
  return GP_OK;
}

int gp_lml_grad_batched(gp_ctx* c, int32_t n_inst, const int64_t* offsets, const double* x, const double* y,
                        const double* h, const gp_opts* o, double* lml, double* grad, gp_info* info) {
  if (!c || !o || n_inst < 0 || (n_inst > 0 && (!offsets || !h || !lml))) return GP_ERR_INVALID_ARG;
  GP_CHECK(check_opts(o, true));
  if (info) memset(info, 0, sizeof(*info));
  if (n_inst == 0) return GP_OK;
  for (int32_t q = 0; q < n_inst; ++q)
    if (offsets[q] < 0 || offsets[q + 1] < offsets[q]) return GP_ERR_INVALID_ARG;
  GP_CUDA(cudaSetDevice(c->device));
  const int64_t P = (int64_t)c->nb * (c->dim + 2) + 3 + (c->core == GP_CORE_SQEXP ? 1 : 0);
  int nw = o->batch_workers > 0 ? o->batch_workers : 8;
  if (nw > n_inst) nw = n_inst;
  // the CG runs of the instances as grouped launches, unless the options ask
  // for what those do not cover (FP64, the Taylor series, injected faults, a
  // product form other than the wide cp.async one) or for the worker streams
  const int spmm_flags = o->flags & (GP_FLAG_SPMM_CPASYNC | GP_FLAG_SPMM_TMA | GP_FLAG_SPMM_TMA_WIDE |
                                     GP_FLAG_SPMM_CPASYNC_WIDE | GP_FLAG_SPMM_WINDOW);
  const bool grouped = !(o->flags & GP_FLAG_BATCH_STREAMS) && o->precision == GP_FP32_MIXED &&
                       !(o->flags & (GP_FLAG_LOGDET_TAYLOR | GP_FLAG_FAULT_OOM | GP_FLAG_FAULT_NOT_SPD |
                                     GP_FLAG_FAULT_NAN)) &&
                       (spmm_flags == 0 || spmm_flags == GP_FLAG_SPMM_CPASYNC_WIDE);
  // grouped: one worker context per instance of a wave; else one per worker
  const int nctx = grouped ? (n_inst < kBatchWave ? n_inst : kBatchWave) : nw;
  // worker contexts: own stream, workspace and CG graphs; kept for later calls
  while ((int)c->workers.size() < nctx) {
    cudaStream_t s = nullptr;
    GP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    const gp_kernel_desc d{c->dim, c->n1, c->n2, c->beta, c->core};
    gp_ctx* w = nullptr;
    const int st = gp_create(&w, &d, c->device, s);
    if (st != GP_OK) {
      cudaStreamDestroy(s);
      return st;
    }
    w->owned_stream = s;
    c->workers.push_back(w);
  }
  // the workers start after everything already queued on the context stream
  // (the inputs may be produced there)
  cudaEvent_t ready = nullptr;
  GP_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  GP_CUDA(cudaEventRecord(ready, c->stream));
  for (int wi = 0; wi < nctx; ++wi) GP_CUDA(cudaStreamWaitEvent(c->workers[wi]->stream, ready, 0));
  cudaEventDestroy(ready);
  // largest instances first, so the tail is short
  std::vector<int32_t> order(n_inst);
  for (int32_t q = 0; q < n_inst; ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return offsets[a + 1] - offsets[a] > offsets[b + 1] - offsets[b];
  });
  std::vector<double> lml_h(n_inst, 0.0), grad_h(grad ? (size_t)n_inst * P : 0);
  std::vector<gp_info> infos(n_inst);
  std::vector<int> status(n_inst, GP_OK);
  std::atomic<bool> abort{false};
  auto failed = [](int s) { return s != GP_OK && s != GP_ERR_NOT_CONVERGED; };
  // fn(t, wi) for t < count, pulled by nw host threads (wi: the thread)
  auto pool = [&](int32_t count, const auto& fn) {
    std::atomic<int32_t> next{0};
    auto work = [&](int wi) {
      cudaSetDevice(c->device);
      for (;;) {
        const int32_t t = next.fetch_add(1);
        if (t >= count || abort.load()) break;
        fn(t, wi);
      }
    };
    std::vector<std::thread> threads;
    for (int wi = 1; wi < nw; ++wi) threads.emplace_back(work, wi);
    work(0);
    for (std::thread& t : threads) t.join();
  };
  auto xs = [&](int32_t q) { return x ? x + offsets[q] * c->dim : nullptr; };
  auto ysrc = [&](int32_t q) { return y ? y + offsets[q] : nullptr; };
  auto gout = [&](int32_t q) { return grad ? grad_h.data() + (size_t)q * P : nullptr; };
  const int64_t launches0 = c->launches;
  if (!grouped) {
    // each instance on its own through evaluate, on the pulling thread's context
    pool(n_inst, [&](int32_t t, int wi) {
      const int32_t q = order[t];
      status[q] = evaluate(c->workers[wi], xs(q), ysrc(q), offsets[q + 1] - offsets[q], h + q * P, o, &lml_h[q],
                           gout(q), &infos[q]);
      if (failed(status[q])) abort.store(true);
    });
  } else {
    for (int32_t w0 = 0; w0 < n_inst && !abort.load(); w0 += nctx) {
      const int32_t nwv = n_inst - w0 < nctx ? n_inst - w0 : nctx;
      // instance j of the wave: order[w0 + j] on worker context j
      std::vector<EvalRun> runs(nwv);
      pool(nwv, [&](int32_t j, int) {
        const int32_t q = order[w0 + j];
        status[q] = eval_front(c->workers[j], xs(q), ysrc(q), offsets[q + 1] - offsets[q], h + q * P, o, &runs[j]);
        if (failed(status[q])) abort.store(true);
      });
      if (abort.load()) break;
      // the CG runs of the wave as grouped launches on the context stream
      const int nv = runs[0].nv, k = runs[0].k, kp = runs[0].kp;
      std::vector<int32_t> pcj, plainj;
      for (int32_t j = 0; j < nwv; ++j) {
        const gp_ctx* w = c->workers[j];
        if (w->n_act > 0) (w->pc_block > 0 ? pcj : plainj).push_back(j);
      }
      auto run_group = [&](const std::vector<int32_t>& js, int m_hist, int max_iter, int check_every, bool use_pc,
                           bool warm, bool lanczos) -> int {
        const size_t m = js.size();
        if (m == 0) return GP_OK;
        std::vector<gp_ctx*> cs(m);
        std::vector<const double*> ys(m);
        std::vector<int> it(m), st(m);
        std::vector<double> rel(m);
        for (size_t i = 0; i < m; ++i) {
          cs[i] = c->workers[js[i]];
          ys[i] = runs[js[i]].yd;
        }
        GP_CHECK(gp::cg_run_group(c, cs.data(), (int)m, k, kp, ys.data(), nv, o->seed, m_hist, max_iter,
                                  o->cg_rtol, check_every, use_pc, warm, it.data(), rel.data(), st.data()));
        for (size_t i = 0; i < m; ++i) {
          EvalRun& r = runs[js[i]];
          const int32_t q = order[w0 + js[i]];
          if (lanczos) {
            r.lanczos_iters = it[i];
            if (failed(st[i])) status[q] = st[i];
          } else {
            r.iters = it[i];
            r.max_rel = rel[i];
            r.cg_status = st[i];
          }
        }
        return GP_OK;
      };
      const int L = o->lanczos_steps;
      int gst = GP_OK;
      // one plain run per instance: its first lanczos_steps coefficients feed SLQ
      if (gst == GP_OK) gst = run_group(plainj, L, o->max_iter, o->check_every, false, false, false);
      if (gst == GP_OK && !pcj.empty()) {
        // the Lanczos run of lanczos_steps plain iterations, SLQ on each
        // instance's side stream, then the preconditioned solves from the
        // Lanczos iterate (as eval_solve does for one instance)
        gst = run_group(pcj, L, L, L, false, false, true);
        std::vector<int32_t> ok;
        for (int32_t j : pcj) {
          const int32_t q = order[w0 + j];
          if (gst == GP_OK && !failed(status[q])) status[q] = gp::slq(c->workers[j], nv, kp, true);
          if (!failed(status[q])) ok.push_back(j);
        }
        if (gst == GP_OK) gst = run_group(ok, 0, o->max_iter, o->check_every, true, true, false);
        for (int32_t j : ok) {
          const int32_t q = order[w0 + j];
          const int jst = gp::slq_join(c->workers[j]);
          if (jst != GP_OK) status[q] = jst;
        }
      }
      if (gst != GP_OK) return gst;
      for (int32_t j = 0; j < nwv; ++j)
        if (failed(status[order[w0 + j]])) abort.store(true);
      if (abort.load()) break;
      pool(nwv, [&](int32_t j, int) {
        const int32_t q = order[w0 + j];
        status[q] = eval_back(c->workers[j], o, runs[j], &lml_h[q], gout(q), &infos[q]);
        if (failed(status[q])) abort.store(true);
      });
    }
  }
  int result = GP_OK;
  for (int32_t q = 0; q < n_inst; ++q) {
    if (status[q] != GP_OK && status[q] != GP_ERR_NOT_CONVERGED) return status[q];
    if (status[q] != GP_OK) result = status[q];
  }
  if (gp::is_device_ptr(lml)) {
    GP_CUDA(cudaMemcpy(lml, lml_h.data(), (size_t)n_inst * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    memcpy(lml, lml_h.data(), (size_t)n_inst * sizeof(double));
  }
  if (grad) {
    if (gp::is_device_ptr(grad))
      GP_CUDA(cudaMemcpy(grad, grad_h.data(), grad_h.size() * sizeof(double), cudaMemcpyHostToDevice));
    else
      memcpy(grad, grad_h.data(), grad_h.size() * sizeof(double));
  }
  if (info) {
    for (int32_t q = 0; q < n_inst; ++q) {
      const gp_info& inf = infos[q];
      info->n += inf.n;
      info->n_active += inf.n_active;
      info->nnz += inf.nnz;
      info->iters = inf.iters > info->iters ? inf.iters : info->iters;
      info->t_assemble_ms += inf.t_assemble_ms;
      info->t_solve_ms += inf.t_solve_ms;
      info->t_grad_ms += inf.t_grad_ms;
      info->launches += inf.launches;
      info->lanczos_iters = inf.lanczos_iters > info->lanczos_iters ? inf.lanczos_iters : info->lanczos_iters;
      info->precond_block = inf.precond_block > info->precond_block ? inf.precond_block : info->precond_block;
      info->n_spmm += inf.n_spmm;
      info->t_spmm_kernel_ms += inf.t_spmm_kernel_ms;
      info->kp = inf.kp;
      // the instances' common SpMM form, -1 if they differ
      info->spmm_variant = q == 0 || inf.spmm_variant == info->spmm_variant ? inf.spmm_variant : -1;
    }
    info->launches += c->launches - launches0;  // the grouped launches
  }
  return result;
}

const char* gp_status_string(int s) {
  switch (s) {
    case GP_OK: return "ok";
    case GP_ERR_INVALID_ARG: return "invalid argument";
    case GP_ERR_CUDA: return "CUDA runtime error";
    case GP_ERR_OOM: return "device out of memory";
    case GP_ERR_NOT_CONVERGED: return "CG did not converge within max_iter";
    case GP_ERR_NOT_SPD: return "CG breakdown: matrix not positive definite";
    case GP_ERR_TIMEOUT: return "bounded device wait timed out";
    case GP_ERR_NOT_ASSEMBLED: return "no assembled matrix";
    case GP_ERR_UNSUPPORTED: return "size above a compiled limit";
    default: return "unknown status";
  }
}

}  // extern "C"
