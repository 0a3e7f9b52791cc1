// Q = Khat P, the product that dominates every CG iteration (Sec. 2.5: each
// conjugate-gradient step multiplies K by the search directions; here one
// product serves y and all probe columns at once).  Khat is stored as an 8x1
// block CSR (eight consecutive Morton-ordered rows share one column index and
// one 32-byte run of values); P and Q are N_act x kp FP32, row-major.
//
// Two ways of feeding the product, chosen per matrix by a small autotuner
// (spmm_select) or forced through gp_opts.flags:
//   * GP_SPMM_CPASYNC: each warp copies the P rows and block values of its
//     next chunk of blocks into shared memory with per-lane cp.async;
//   * GP_SPMM_TMA / GP_SPMM_TMA_WIDE: the tensor-memory accelerator fills the
//     same stage: tile::gather4 loads bring four P rows per request (their row
//     indices are the chunk's block columns) and one bulk copy brings the
//     chunk's block values, all completing on the stage's mbarrier.  The
//     load/store unit then serves only the shared-memory reads of the
//     arithmetic.  The wide form gives each lane LW float4 columns of P, so
//     that one warp step applies ten blocks instead of three and the block
//     values are read from shared memory a third as often;
//   * GP_SPMM_CPASYNC_WIDE: the per-lane cp.async stage with the wide lanes.
// Every form computes, per output element, a sum of the same products; the
// forms differ only in the order of the FP32 additions.
#include <cuda.h>

#include <map>
#include <mutex>
#include <tuple>

#include "gp_internal.cuh"
#include "async.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;

// A: Q = Khat P on the 8x1 block CSR.  Each CTA owns a contiguous run of
// block rows holding an equal share of the stored blocks; its warps take the
// rows round-robin (neighbouring block rows gather overlapping P rows close
// together in time, while they are in L2), and each warp streams its rows'
// blocks in chunks through a double-buffered shared-memory stage: while the
// warp computes chunk c, cp.async copies the P rows (kp floats) and the 8
// values of chunk c+1 into the other buffer, and the column indices of chunk
// c+2 are already being loaded.  Compute: the warp's lanes form NG = 32/G
// groups of G lanes (one float4 of the kp = 4G columns per lane); a group
// takes every NG-th block of the chunk and applies its P row to the 8 rows
// of the block row (8 float4 accumulators per lane).  A chunk holds
// NG floor(32 / NG) blocks, a whole number of warp steps, so that no step
// multiplies an empty slot in the middle of a block row.
// Smallest block row b in [0, nblk] whose first stored block is >= target
// (brp ascending, brp[nblk] = total).  Every block row then belongs to
// exactly one CTA's share.
__device__ inline int64_t first_row_at_or_after(const int64_t* __restrict__ brp, int64_t nblk, int64_t target) {
  int64_t lo = 0, hi = nblk;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(brp + mid) < target) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

constexpr int kSpmmThreads = 128;
constexpr int kSpmmWarps = kSpmmThreads / 32;
constexpr int kBR = 8;
constexpr int kChunk = 32;

// The stage copies bypass the L1 (.cg): allocating the gathered P rows there
// as well cost more L1 throughput than its hits saved.
__device__ inline void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Position of a chunk in the warp's stream: block row bb, first block base.
struct ChunkPos {
  int64_t bb, base;
};

template <int CH = kChunk>
__device__ inline ChunkPos next_chunk(ChunkPos c, const int64_t* __restrict__ brp, int64_t b1) {
  const int64_t e = __ldg(brp + c.bb + 1);
  if (c.base + CH < e) return {c.bb, c.base + CH};
  const int64_t nb = c.bb + kSpmmWarps;
  if (nb >= b1) return {b1, 0};
  return {nb, __ldg(brp + nb)};
}

template <int G>
__global__ void __launch_bounds__(kSpmmThreads) k_bspmm_f32(int64_t n, int64_t nblk,
                                                            const int64_t* __restrict__ brp,
                                                            const int32_t* __restrict__ bcol,
                                                            const float4* __restrict__ bval,
                                                            const float4* __restrict__ P, float4* __restrict__ Q,
                                                            double* __restrict__ part, gp::CgState* st,
    gp::Group g) {
  int bx = blockIdx.x, gx = gridDim.x;
  if (g.inst) {
    const gp::GInst* I = gpd::group_cta(g, gp::kGSpmm, bx, gx);
    n = I->n;
    nblk = I->nblk;
    brp = I->brp;
    bcol = I->bcol;
    bval = I->bval;
    P = I->P;
    Q = I->Q;
    part = I->part_a;
    st = I->st;
  }
  const int it = st->iter;
  if (st->fin[it & 1]) return;
  constexpr int NG = 32 / G;
  constexpr int KP = 4 * G;
  constexpr int kStage = kChunk * (KP + kBR);  // floats per stage buffer
  // a chunk holds a whole number of warp steps; lane l copies piece l % G of
  // entry l / G of each group of EPI entries
  constexpr int CH = NG * (kChunk / NG);
  constexpr int kSteps = CH / NG;
  constexpr int EPI = 32 / G;
  constexpr int NIS = (CH + EPI - 1) / EPI;
  extern __shared__ float4 smem_f4[];
  float* stage = (float*)smem_f4 + (size_t)(threadIdx.x >> 5) * 2 * kStage;
  __shared__ double sh[kSpmmWarps][KP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane - grp * G;
  const bool act = grp < NG;
  const bool lcopy = grp < EPI;  // EPI == NG: the copy layout is the compute layout
  gpd::Dot2 pq0, pq1, pq2, pq3;
  // Work split by stored blocks, not by block rows (cluster cores hold many
  // times more blocks per row than the background).
  const int64_t nent = brp[nblk];
  const int64_t cb0 = first_row_at_or_after(brp, nblk, nent * bx / gx);
  const int64_t b1 = first_row_at_or_after(brp, nblk, nent * (bx + 1) / gx);
  const int64_t b0 = cb0 + w;
  if (b0 < b1) {
    // stage a chunk: consecutive lanes copy consecutive 16-byte pieces of the
    // same P row (G pieces per row, so one copy instruction covers about 32/G
    // rows), then the chunk's block values (2 float4 each, contiguous)
    auto issue = [&](ChunkPos c, int jl, int buf) {
      if (c.bb < b1) {
        const int64_t e = __ldg(brp + c.bb + 1);
        const int cnt = (int)min((int64_t)CH, e - c.base);
        float* dst = stage + buf * kStage;
        float* dl = dst + grp * KP + 4 * gl;
        const float4* pl = P + gl;
#pragma unroll
        for (int i = 0; i < NIS; ++i) {
          const int ent = i * EPI + grp;
          const int j = __shfl_sync(kFull, jl, ent < 32 ? ent : 31);
          if (lcopy && ent < cnt) cp_async16(dl + i * EPI * KP, pl + (int64_t)j * G);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int q = lane + 32 * i;
          if (q < 2 * cnt) cp_async16(dst + kChunk * KP + 4 * q, bval + 2 * c.base + q);
        }
      }
      cp_async_commit();
    };
    auto col_of = [&](ChunkPos c) -> int {
      if (c.bb >= b1) return 0;
      const int64_t idx = c.base + lane;
      return lane < CH && idx < __ldg(brp + c.bb + 1) ? __ldg(bcol + idx) : 0;
    };
    ChunkPos cur{b0, __ldg(brp + b0)};
    ChunkPos nx1 = next_chunk<CH>(cur, brp, b1);
    issue(cur, col_of(cur), 0);
    int j1 = col_of(nx1);
    // accumulators as float2 pairs (columns x,y and z,w of the lane's float4)
    // for the packed two-wide FP32 FMA, which rounds each half like fmaf
    float2 acc[2 * kBR];
#pragma unroll
    for (int r = 0; r < 2 * kBR; ++r) acc[r] = make_float2(0.f, 0.f);
    int buf = 0;
    while (cur.bb < b1) {
      const ChunkPos nx2 = nx1.bb < b1 ? next_chunk<CH>(nx1, brp, b1) : nx1;
      issue(nx1, j1, buf ^ 1);            // copies of chunk c+1 in flight
      const int j2 = col_of(nx2);          // indices of chunk c+2 in flight
      cp_async_wait<1>();                  // chunk c has landed
      __syncwarp();
      const int64_t e = __ldg(brp + cur.bb + 1);
      const int cnt = (int)min((int64_t)CH, e - cur.base);
      const float* sp = stage + buf * kStage;
      const float* sv = sp + kChunk * KP;
#pragma unroll 2
      for (int t = 0; t < kSteps; ++t) {
        const int src = t * NG + grp;
        if (act && src < cnt) {
          const float4 pj = *(const float4*)(sp + src * KP + 4 * gl);
          const float4 v0 = *(const float4*)(sv + src * kBR);
          const float4 v1 = *(const float4*)(sv + src * kBR + 4);
          const float vv[kBR] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
          const float2 plo = make_float2(pj.x, pj.y), phi = make_float2(pj.z, pj.w);
#pragma unroll
          for (int r = 0; r < kBR; ++r) {
            const float2 v2 = make_float2(vv[r], vv[r]);
            acc[2 * r] = __ffma2_rn(v2, plo, acc[2 * r]);
            acc[2 * r + 1] = __ffma2_rn(v2, phi, acc[2 * r + 1]);
          }
        }
      }
      __syncwarp();  // buffer `buf` may be refilled from the next iteration on
      if (cur.base + CH >= e) {
        // last chunk of block row cur.bb: group 0 adds the other groups' sums
#pragma unroll
        for (int r = 0; r < 2 * kBR; ++r) {
          const float2 q0 = acc[r];
#pragma unroll
          for (int g2 = 1; g2 < NG; ++g2) {
            const int src = gl + g2 * G;
            acc[r].x += __shfl_sync(kFull, q0.x, src);
            acc[r].y += __shfl_sync(kFull, q0.y, src);
          }
        }
        if (grp == 0) {
#pragma unroll
          for (int r = 0; r < kBR; ++r) {
            const int64_t row = cur.bb * kBR + r;
            if (row < n) {
              const float4 qv = make_float4(acc[2 * r].x, acc[2 * r].y, acc[2 * r + 1].x, acc[2 * r + 1].y);
              Q[row * G + gl] = qv;
              const float4 pp = __ldg(P + row * G + gl);
              pq0.add(pp.x, qv.x);
              pq1.add(pp.y, qv.y);
              pq2.add(pp.z, qv.z);
              pq3.add(pp.w, qv.w);
            }
          }
        }
#pragma unroll
        for (int r = 0; r < 2 * kBR; ++r) acc[r] = make_float2(0.f, 0.f);
      }
      cur = nx1;
      nx1 = nx2;
      j1 = j2;
      buf ^= 1;
    }
    cp_async_wait<0>();
  }
  if (grp == 0) {
    sh[w][4 * gl + 0] = pq0.value();
    sh[w][4 * gl + 1] = pq1.value();
    sh[w][4 * gl + 2] = pq2.value();
    sh[w][4 * gl + 3] = pq3.value();
  }
  __syncthreads();
  if (threadIdx.x < KP) {
    double t = 0.0;
    for (int ww = 0; ww < kSpmmWarps; ++ww) t += sh[ww][threadIdx.x];
    part[(int64_t)bx * KP + threadIdx.x] = t;
  }
}


// ---------------------------------------------------------------- TMA form
// Stage layout of one buffer: the chunk's P rows in groups of four (one
// gather4 each, padded to 128 bytes), then its 32 blocks' values.
constexpr int tma_group_bytes(int kq) { return (64 * kq + 127) / 128 * 128; }
constexpr int tma_stage_bytes(int kq) { return (kChunk / 4) * tma_group_bytes(kq) + kChunk * kBR * 4; }
// Stage buffers per warp (NS - 1 chunks in flight while one is computed).
// Two: on the 1M-point mixture (kp = 36) a third buffer made the TMA forms
// slower (narrow 462 -> 563 us, wide 422 -> 450 us per launch), since it costs
// a CTA per SM and the gather4 requests, not their latency, set the pace.
constexpr int tma_stages(int) { return 2; }
constexpr size_t tma_smem_bytes(int kq) {
  return (size_t)kSpmmWarps * tma_stages(kq) * tma_stage_bytes(kq) + 128;
}
// float4 columns per lane of the wide form
constexpr int wide_lw(int kq) { return (kq % 3 == 0 && kq >= 6) ? 3 : (kq % 2 == 0 && kq >= 4) ? 2 : 1; }
// rows per pass of the wide form's cross-group sum (its scratch is one stage buffer)
constexpr int wide_rows_per_pass(int ng, int kq) {
  return ng * 8 * kq * 16 <= tma_stage_bytes(kq)   ? 8
         : ng * 4 * kq * 16 <= tma_stage_bytes(kq) ? 4
         : ng * 2 * kq * 16 <= tma_stage_bytes(kq) ? 2
                                                    : 1;
}

// Q = Khat P with TMA-filled stages.  KQ = kp / 4 float4 columns; each lane
// holds LW of them for the 8 rows of a block row, a group of G = KQ / LW lanes
// applies one block, NG = 32 / G groups work on different blocks of the same
// block row.  Work split, chunking and the p^T q partials as in k_bspmm_f32;
// each warp keeps NS - 1 chunks in flight in a ring of NS stage buffers.  A
// bounded wait that gives up records GP_ERR_TIMEOUT in the CG state, waits
// (bounded) for the copies it issued, and leaves.
template <int KQ, int LW>
__global__ void __launch_bounds__(kSpmmThreads) k_bspmm_tma(int64_t n, int64_t nblk,
                                                            const int64_t* __restrict__ brp,
                                                            const int32_t* __restrict__ bcol,
                                                            const float4* __restrict__ bval,
                                                            const __grid_constant__ CUtensorMap tmP,
                                                            const float4* __restrict__ P, float4* __restrict__ Q,
                                                            double* __restrict__ part, gp::CgState* st) {
  const int it = st->iter;
  if (st->fin[it & 1]) return;
  static_assert(KQ % LW == 0, "LW must divide KQ");
  constexpr int G = KQ / LW;
  constexpr int NG = 32 / G;
  constexpr int KP = 4 * KQ;
  constexpr int ROWB = 16 * KQ;
  constexpr int GB = tma_group_bytes(KQ);
  constexpr int PB = (kChunk / 4) * GB;
  constexpr int SB = tma_stage_bytes(KQ);
  constexpr int NS = tma_stages(KQ);
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_s[kSpmmWarps][NS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned char* stage =
      (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127) + (size_t)w * NS * SB;
  uint64_t* bar = bar_s[w];
  const int grp = lane / G, gl = lane - grp * G;
  const bool act = grp < NG;
  // lanes that own an output float4 slot for the p^T q partials
  constexpr int M = 32 / KQ;
  const int slot = LW == 1 ? (lane < KQ ? lane : -1) : (lane < M * KQ ? lane % KQ : -1);
  gpd::Dot2 pq0, pq1, pq2, pq3;
  if (lane == 0) {
    for (int b = 0; b < NS; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
  }
  __syncwarp();
  const int64_t nent = brp[nblk];
  const int64_t cb0 = first_row_at_or_after(brp, nblk, nent * blockIdx.x / gridDim.x);
  const int64_t b1 = first_row_at_or_after(brp, nblk, nent * (blockIdx.x + 1) / gridDim.x);
  const int64_t b0 = cb0 + w;
  unsigned phase = 0, inflight = 0;
  if (b0 < b1) {
    // chunk c into buffer buf: lane g < ceil(cnt/4) gathers entries 4g..4g+3
    // (entries past cnt repeat column 0, a valid row, and are not used); one
    // lane copies the values.  The arrival with the byte count comes first.
    auto issue = [&](ChunkPos c, int jl, int buf) {
      if (c.bb >= b1) return;
      const int64_t e = __ldg(brp + c.bb + 1);
      const int cnt = (int)min((int64_t)kChunk, e - c.base);
      const int ng4 = (cnt + 3) >> 2;
      const int q0 = 4 * (lane & 7);
      const int r0 = __shfl_sync(kFull, jl, q0), r1 = __shfl_sync(kFull, jl, q0 + 1);
      const int r2 = __shfl_sync(kFull, jl, q0 + 2), r3 = __shfl_sync(kFull, jl, q0 + 3);
      unsigned char* dst = stage + buf * SB;
      if (lane == 0) mbar_arrive_expect(&bar[buf], (unsigned)(ng4 * 4 * ROWB + cnt * kBR * 4));
      __syncwarp();
      if (lane < ng4) tma_gather4(dst + lane * GB, &tmP, r0, r1, r2, r3, &bar[buf]);
      if (lane == 31) bulk_to_smem(dst + PB, bval + 2 * c.base, (unsigned)(cnt * kBR * 4), &bar[buf]);
      inflight |= 1u << buf;
    };
    auto col_of = [&](ChunkPos c) -> int {
      if (c.bb >= b1) return 0;
      const int64_t idx = c.base + lane;
      return idx < __ldg(brp + c.bb + 1) ? __ldg(bcol + idx) : 0;
    };
    // chunk ring: pos[i] is chunk c+i; chunks c .. c+NS-2 are in flight or
    // landed, the column indices of chunk c+NS-1 are in jn
    ChunkPos pos[NS + 1];
    pos[0] = ChunkPos{b0, __ldg(brp + b0)};
#pragma unroll
    for (int i = 1; i <= NS; ++i) pos[i] = pos[i - 1].bb < b1 ? next_chunk(pos[i - 1], brp, b1) : pos[i - 1];
#pragma unroll
    for (int i = 0; i < NS - 1; ++i) issue(pos[i], col_of(pos[i]), i);
    int jn = col_of(pos[NS - 1]);
    float2 acc[kBR][2 * LW];
#pragma unroll
    for (int r = 0; r < kBR; ++r)
#pragma unroll
      for (int u = 0; u < 2 * LW; ++u) acc[r][u] = make_float2(0.f, 0.f);
    int buf = 0;
    bool failed = false;
    while (pos[0].bb < b1) {
      const ChunkPos cur = pos[0];
      issue(pos[NS - 1], jn, buf + NS - 1 < NS ? buf + NS - 1 : buf - 1);  // chunk c+NS-1 in flight
      jn = col_of(pos[NS]);                                                // its successor's indices
      const bool ok = __all_sync(kFull, mbar_wait(&bar[buf], (phase >> buf) & 1u));
      if (!ok) {
        failed = true;
        break;
      }
      phase ^= 1u << buf;
      inflight &= ~(1u << buf);
      const int64_t e = __ldg(brp + cur.bb + 1);
      const int cnt = (int)min((int64_t)kChunk, e - cur.base);
      const unsigned char* sp = stage + buf * SB;
      const float* sv = (const float*)(sp + PB);
      constexpr int kSteps = (kChunk + NG - 1) / NG;
#pragma unroll 2
      for (int t = 0; t < kSteps; ++t) {
        const int src = t * NG + grp;
        if (act && src < cnt) {
          const float* prow = (const float*)(sp + (src >> 2) * GB + (src & 3) * ROWB) + 4 * LW * gl;
          float4 pj[LW];
#pragma unroll
          for (int u = 0; u < LW; ++u) pj[u] = *(const float4*)(prow + 4 * u);
          const float4 v0 = *(const float4*)(sv + src * kBR);
          const float4 v1 = *(const float4*)(sv + src * kBR + 4);
          const float vv[kBR] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
          for (int r = 0; r < kBR; ++r) {
            const float2 v2 = make_float2(vv[r], vv[r]);
#pragma unroll
            for (int u = 0; u < LW; ++u) {
              acc[r][2 * u] = __ffma2_rn(v2, make_float2(pj[u].x, pj[u].y), acc[r][2 * u]);
              acc[r][2 * u + 1] = __ffma2_rn(v2, make_float2(pj[u].z, pj[u].w), acc[r][2 * u + 1]);
            }
          }
        }
      }
      __syncwarp();
      if (cur.base + kChunk >= e) {
        // last chunk of block row cur.bb: add the NG groups' sums, write Q
        if constexpr (LW == 1) {
#pragma unroll
          for (int r = 0; r < kBR; ++r)
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const float2 q0 = acc[r][u];
#pragma unroll
              for (int g2 = 1; g2 < NG; ++g2) {
                const int src = gl + g2 * G;
                acc[r][u].x += __shfl_sync(kFull, q0.x, src);
                acc[r][u].y += __shfl_sync(kFull, q0.y, src);
              }
            }
          if (grp == 0) {
#pragma unroll
            for (int r = 0; r < kBR; ++r) {
              const int64_t row = cur.bb * kBR + r;
              if (row < n) {
                const float4 qv = make_float4(acc[r][0].x, acc[r][0].y, acc[r][1].x, acc[r][1].y);
                Q[row * KQ + gl] = qv;
                const float4 pp = __ldg(P + row * KQ + gl);
                pq0.add(pp.x, qv.x);
                pq1.add(pp.y, qv.y);
                pq2.add(pp.z, qv.z);
                pq3.add(pp.w, qv.w);
              }
            }
          }
        } else {
          // through the stage buffer just consumed: groups write their
          // partial rows, then lane l sums slot l % KQ of rows l / KQ + M i
          constexpr int RP = wide_rows_per_pass(NG, KQ);
          float4* scr = (float4*)(stage + buf * SB);
#pragma unroll
          for (int r0 = 0; r0 < kBR; r0 += RP) {
            if (act) {
#pragma unroll
              for (int r = 0; r < RP; ++r)
#pragma unroll
                for (int u = 0; u < LW; ++u)
                  scr[(grp * RP + r) * KQ + gl * LW + u] = make_float4(
                      acc[r0 + r][2 * u].x, acc[r0 + r][2 * u].y, acc[r0 + r][2 * u + 1].x, acc[r0 + r][2 * u + 1].y);
            }
            __syncwarp();
            if (slot >= 0) {
              for (int r = lane / KQ; r < RP; r += M) {
                float4 s = scr[r * KQ + slot];
                for (int g2 = 1; g2 < NG; ++g2) {
                  const float4 t = scr[(g2 * RP + r) * KQ + slot];
                  s.x += t.x;
                  s.y += t.y;
                  s.z += t.z;
                  s.w += t.w;
                }
                const int64_t row = cur.bb * kBR + r0 + r;
                if (row < n) {
                  Q[row * KQ + slot] = s;
                  const float4 pp = __ldg(P + row * KQ + slot);
                  pq0.add(pp.x, s.x);
                  pq1.add(pp.y, s.y);
                  pq2.add(pp.z, s.z);
                  pq3.add(pp.w, s.w);
                }
              }
            }
            __syncwarp();
          }
          // these generic writes precede the next TMA fill of the buffer
          fence_proxy_async_smem();
          __syncwarp();
        }
#pragma unroll
        for (int r = 0; r < kBR; ++r)
#pragma unroll
          for (int u = 0; u < 2 * LW; ++u) acc[r][u] = make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int i = 0; i < NS; ++i) pos[i] = pos[i + 1];
      pos[NS] = pos[NS].bb < b1 ? next_chunk(pos[NS], brp, b1) : pos[NS];
      buf = buf + 1 < NS ? buf + 1 : 0;
    }
    if (failed) {
      if (lane == 0) atomicCAS(&st->status, GP_OK, GP_ERR_TIMEOUT);
      // the copies this warp issued must land before its shared memory goes
      for (int b = 0; b < NS; ++b)
        if (inflight & (1u << b)) mbar_wait(&bar[b], (phase >> b) & 1u);
    }
  }
  // per-lane partials in the warp's first stage buffer (every copy into it
  // has landed), then summed per column in a fixed order
  double* shp = (double*)stage;  // [32][4] of this warp
  __syncwarp();
  shp[4 * lane + 0] = slot >= 0 ? pq0.value() : 0.0;
  shp[4 * lane + 1] = slot >= 0 ? pq1.value() : 0.0;
  shp[4 * lane + 2] = slot >= 0 ? pq2.value() : 0.0;
  shp[4 * lane + 3] = slot >= 0 ? pq3.value() : 0.0;
  __syncthreads();
  if (threadIdx.x < KP) {
    const int q = threadIdx.x >> 2, cc = threadIdx.x & 3;
    const unsigned char* base = (const unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    double t = 0.0;
    for (int ww = 0; ww < kSpmmWarps; ++ww)
      for (int l = 0; l < 32; ++l) {
        const int sl = LW == 1 ? (l < KQ ? l : -1) : (l < M * KQ ? l % KQ : -1);
        if (sl == q) t += ((const double*)(base + (size_t)ww * NS * SB))[4 * l + cc];
      }
    part[(int64_t)blockIdx.x * KP + threadIdx.x] = t;
  }
}

// ---------------------------------------------------------------- wide cp.async form
// The per-lane cp.async stage of k_bspmm_f32 with the lane layout of the wide
// TMA form: each lane holds LW float4 columns for the 8 rows of a block row,
// so a warp step applies NG = 32 / (KQ / LW) blocks (10 at kp = 36) and the
// block values are read from shared memory a third as often.  The groups'
// partial rows are added through the stage buffer just consumed, RP rows per
// pass (the buffer holds kChunk (KP + 8) floats).
constexpr int cpw_rows_per_pass(int ng, int kq) {
  return ng * 8 * kq * 4 <= kChunk * (4 * kq + kBR)   ? 8
         : ng * 4 * kq * 4 <= kChunk * (4 * kq + kBR) ? 4
         : ng * 2 * kq * 4 <= kChunk * (4 * kq + kBR) ? 2
                                                       : 1;
}

template <int KQ, int LW>
__global__ void __launch_bounds__(kSpmmThreads) k_bspmm_f32w(int64_t n, int64_t nblk,
                                                             const int64_t* __restrict__ brp,
                                                             const int32_t* __restrict__ bcol,
                                                             const float4* __restrict__ bval,
                                                             const float4* __restrict__ P, float4* __restrict__ Q,
                                                             double* __restrict__ part, gp::CgState* st,
    gp::Group g) {
  int bx = blockIdx.x, gx = gridDim.x;
  if (g.inst) {
    const gp::GInst* I = gpd::group_cta(g, gp::kGSpmm, bx, gx);
    n = I->n;
    nblk = I->nblk;
    brp = I->brp;
    bcol = I->bcol;
    bval = I->bval;
    P = I->P;
    Q = I->Q;
    part = I->part_a;
    st = I->st;
  }
  const int it = st->iter;
  if (st->fin[it & 1]) return;
  static_assert(KQ % LW == 0 && LW > 1, "wide lanes");
  constexpr int G = KQ / LW;
  constexpr int NG = 32 / G;
  constexpr int KP = 4 * KQ;
  constexpr int kStage = kChunk * (KP + kBR);  // floats per stage buffer
  constexpr int RP = cpw_rows_per_pass(NG, KQ);
  constexpr int M = 32 / KQ;
  // a chunk holds a whole number of warp steps (30 blocks at NG = 10)
  constexpr int CH = NG * (kChunk / NG);
  constexpr int kSteps = CH / NG;
  // copy layout: lane l copies piece l % KQ of entry l / KQ of each group of
  // EPI entries, so its shared-memory offset is fixed for the whole run
  constexpr int EPI = 32 / KQ;
  constexpr int NIS = (CH + EPI - 1) / EPI;
  extern __shared__ float4 smem_f4[];
  float* stage = (float*)smem_f4 + (size_t)(threadIdx.x >> 5) * 2 * kStage;
  __shared__ double shp[kSpmmWarps][32][4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane - grp * G;
  const bool act = grp < NG;
  const int slot = lane < M * KQ ? lane % KQ : -1;
  const int le = lane / KQ, lp = lane - le * KQ;
  const bool lcopy = le < EPI;
  gpd::Dot2 pq0, pq1, pq2, pq3;
  const int64_t nent = brp[nblk];
  const int64_t cb0 = first_row_at_or_after(brp, nblk, nent * bx / gx);
  const int64_t b1 = first_row_at_or_after(brp, nblk, nent * (bx + 1) / gx);
  const int64_t b0 = cb0 + w;
  if (b0 < b1) {
    // stage a chunk as k_bspmm_f32 does: KQ 16-byte pieces per P row, then the
    // chunk's block values
    auto issue = [&](ChunkPos c, int jl, int buf) {
      if (c.bb < b1) {
        const int64_t e = __ldg(brp + c.bb + 1);
        const int cnt = (int)min((int64_t)CH, e - c.base);
        float* dst = stage + buf * kStage;
        float* dl = dst + le * KP + 4 * lp;
        const float4* pl = P + lp;
#pragma unroll
        for (int i = 0; i < NIS; ++i) {
          const int ent = i * EPI + le;
          const int j = __shfl_sync(kFull, jl, ent < 32 ? ent : 31);
          if (lcopy && ent < cnt) cp_async16(dl + i * EPI * KP, pl + (int64_t)j * KQ);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int q = lane + 32 * i;
          if (q < 2 * cnt) cp_async16(dst + kChunk * KP + 4 * q, bval + 2 * c.base + q);
        }
      }
      cp_async_commit();
    };
    auto col_of = [&](ChunkPos c) -> int {
      if (c.bb >= b1) return 0;
      const int64_t idx = c.base + lane;
      return lane < CH && idx < __ldg(brp + c.bb + 1) ? __ldg(bcol + idx) : 0;
    };
    ChunkPos cur{b0, __ldg(brp + b0)};
    ChunkPos nx1 = next_chunk<CH>(cur, brp, b1);
    issue(cur, col_of(cur), 0);
    int j1 = col_of(nx1);
    float2 acc[kBR][2 * LW];
#pragma unroll
    for (int r = 0; r < kBR; ++r)
#pragma unroll
      for (int u = 0; u < 2 * LW; ++u) acc[r][u] = make_float2(0.f, 0.f);
    int buf = 0;
    while (cur.bb < b1) {
      const ChunkPos nx2 = nx1.bb < b1 ? next_chunk<CH>(nx1, brp, b1) : nx1;
      issue(nx1, j1, buf ^ 1);            // copies of chunk c+1 in flight
      const int j2 = col_of(nx2);          // indices of chunk c+2 in flight
      cp_async_wait<1>();                  // chunk c has landed
      __syncwarp();
      const int64_t e = __ldg(brp + cur.bb + 1);
      const int cnt = (int)min((int64_t)CH, e - cur.base);
      const float* sp = stage + buf * kStage;
      const float* sv = sp + kChunk * KP;
#pragma unroll
      for (int t = 0; t < kSteps; ++t) {
        const int src = t * NG + grp;
        if (act && src < cnt) {
          const float* prow = sp + src * KP + 4 * LW * gl;
          float4 pj[LW];
#pragma unroll
          for (int u = 0; u < LW; ++u) pj[u] = *(const float4*)(prow + 4 * u);
          const float4 v0 = *(const float4*)(sv + src * kBR);
          const float4 v1 = *(const float4*)(sv + src * kBR + 4);
          const float vv[kBR] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
          for (int r = 0; r < kBR; ++r) {
            const float2 v2 = make_float2(vv[r], vv[r]);
#pragma unroll
            for (int u = 0; u < LW; ++u) {
              acc[r][2 * u] = __ffma2_rn(v2, make_float2(pj[u].x, pj[u].y), acc[r][2 * u]);
              acc[r][2 * u + 1] = __ffma2_rn(v2, make_float2(pj[u].z, pj[u].w), acc[r][2 * u + 1]);
            }
          }
        }
      }
      __syncwarp();
      if (cur.base + CH >= e) {
        // last chunk of block row cur.bb: groups write their partial rows to
        // the consumed buffer, then lane l sums slot l % KQ of rows l / KQ + M i
        float4* scr = (float4*)(stage + buf * kStage);
#pragma unroll
        for (int r0 = 0; r0 < kBR; r0 += RP) {
          if (act) {
#pragma unroll
            for (int r = 0; r < RP; ++r)
#pragma unroll
              for (int u = 0; u < LW; ++u)
                scr[(grp * RP + r) * KQ + gl * LW + u] = make_float4(
                    acc[r0 + r][2 * u].x, acc[r0 + r][2 * u].y, acc[r0 + r][2 * u + 1].x, acc[r0 + r][2 * u + 1].y);
          }
          __syncwarp();
          if (slot >= 0) {
            for (int r = lane / KQ; r < RP; r += M) {
              float4 sum = scr[r * KQ + slot];
              for (int g2 = 1; g2 < NG; ++g2) {
                const float4 t = scr[(g2 * RP + r) * KQ + slot];
                sum.x += t.x;
                sum.y += t.y;
                sum.z += t.z;
                sum.w += t.w;
              }
              const int64_t row = cur.bb * kBR + r0 + r;
              if (row < n) {
                Q[row * KQ + slot] = sum;
                const float4 pp = __ldg(P + row * KQ + slot);
                pq0.add(pp.x, sum.x);
                pq1.add(pp.y, sum.y);
                pq2.add(pp.z, sum.z);
                pq3.add(pp.w, sum.w);
              }
            }
          }
          __syncwarp();
        }
#pragma unroll
        for (int r = 0; r < kBR; ++r)
#pragma unroll
          for (int u = 0; u < 2 * LW; ++u) acc[r][u] = make_float2(0.f, 0.f);
      }
      cur = nx1;
      nx1 = nx2;
      j1 = j2;
      buf ^= 1;
    }
    cp_async_wait<0>();
  }
  shp[w][lane][0] = slot >= 0 ? pq0.value() : 0.0;
  shp[w][lane][1] = slot >= 0 ? pq1.value() : 0.0;
  shp[w][lane][2] = slot >= 0 ? pq2.value() : 0.0;
  shp[w][lane][3] = slot >= 0 ? pq3.value() : 0.0;
  __syncthreads();
  if (threadIdx.x < KP) {
    const int q = threadIdx.x >> 2, cc = threadIdx.x & 3;
    double t = 0.0;
    for (int ww = 0; ww < kSpmmWarps; ++ww)
      for (int l = 0; l < 32; ++l)
        if ((l < M * KQ ? l % KQ : -1) == q) t += shp[ww][l][cc];
    part[(int64_t)bx * KP + threadIdx.x] = t;
  }
}

// ---------------------------------------------------------------- host side
typedef void (*CpAsyncFn)(int64_t, int64_t, const int64_t*, const int32_t*, const float4*, const float4*, float4*,
                          double*, gp::CgState*, gp::Group);
typedef void (*TmaFn)(int64_t, int64_t, const int64_t*, const int32_t*, const float4*, const CUtensorMap,
                      const float4*, float4*, double*, gp::CgState*);

template <int KQ>
void fill_fns(CpAsyncFn* cp, TmaFn* tn, TmaFn* tw, CpAsyncFn* cw) {
  cp[KQ] = k_bspmm_f32<KQ>;
  tn[KQ] = k_bspmm_tma<KQ, 1>;
  if constexpr (wide_lw(KQ) > 1) {
    tw[KQ] = k_bspmm_tma<KQ, wide_lw(KQ)>;
    cw[KQ] = k_bspmm_f32w<KQ, wide_lw(KQ)>;
  }
}

struct FnTable {
  CpAsyncFn cp[18] = {};
  TmaFn tn[18] = {};
  TmaFn tw[18] = {};
  CpAsyncFn cw[18] = {};
  FnTable() {
    fill_fns<1>(cp, tn, tw, cw);
    fill_fns<2>(cp, tn, tw, cw);
    fill_fns<3>(cp, tn, tw, cw);
    fill_fns<4>(cp, tn, tw, cw);
    fill_fns<5>(cp, tn, tw, cw);
    fill_fns<6>(cp, tn, tw, cw);
    fill_fns<7>(cp, tn, tw, cw);
    fill_fns<8>(cp, tn, tw, cw);
    fill_fns<9>(cp, tn, tw, cw);
    fill_fns<10>(cp, tn, tw, cw);
    fill_fns<11>(cp, tn, tw, cw);
    fill_fns<12>(cp, tn, tw, cw);
    fill_fns<13>(cp, tn, tw, cw);
    fill_fns<14>(cp, tn, tw, cw);
    fill_fns<15>(cp, tn, tw, cw);
    fill_fns<16>(cp, tn, tw, cw);
    fill_fns<17>(cp, tn, tw, cw);
  }
};
const FnTable& fns() {
  static const FnTable t;
  return t;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// Tensor map of P (n rows of kp FP32, row pitch kp * 4 bytes): box = one row.
int encode_p_map(void* out, const float* P, int64_t n, int kp) {
  static_assert(sizeof(CUtensorMap) == sizeof(((gp::SpmmPlan*)nullptr)->tmap), "tensor map size");
  EncodeTiledFn enc = encode_fn();
  if (!enc) return GP_ERR_CUDA;
  if (((uintptr_t)P & 15) || n > ((int64_t)1 << 31) - 1 || kp > 256) return GP_ERR_UNSUPPORTED;
  const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)kp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kp, 1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc((CUtensorMap*)out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)P, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? GP_OK : GP_ERR_CUDA;
}

// Process-wide choice per matrix shape, so that every context (and every
// worker of a batched call) multiplies a given matrix the same way.
struct TuneKey {
  int device, kp;
  int64_t n, nblk, nbent;
  bool operator<(const TuneKey& o) const {
    return std::tie(device, kp, n, nblk, nbent) < std::tie(o.device, o.kp, o.n, o.nblk, o.nbent);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

}  // namespace

namespace gp {

bool spmm_available(int variant, int kp) {
  if (kp % 4 || kp < 4 || kp > 4 * 17) return false;
  const int kq = kp / 4;
  switch (variant) {
    case GP_SPMM_CPASYNC: return true;
    case GP_SPMM_TMA: return encode_fn() != nullptr;
    case GP_SPMM_TMA_WIDE: return encode_fn() != nullptr && fns().tw[kq] != nullptr;
    case GP_SPMM_CPASYNC_WIDE: return fns().cw[kq] != nullptr;
    default: return false;
  }
}

int spmm_plan(gp_ctx* c, int kp, int variant, SpmmPlan* p) {
  if (variant == GP_SPMM_WINDOW) return window_plan(c, kp, p);
  if (!spmm_available(variant, kp)) return GP_ERR_UNSUPPORTED;
  const int kq = kp / 4;
  p->variant = variant;
  p->kp = kp;
  if (variant == GP_SPMM_CPASYNC || variant == GP_SPMM_CPASYNC_WIDE) {
    p->fn = (const void*)(variant == GP_SPMM_CPASYNC ? fns().cp[kq] : fns().cw[kq]);
    p->smem = (size_t)kSpmmWarps * 2 * kChunk * (kp + kBR) * sizeof(float);
  } else {
    p->fn = (const void*)(variant == GP_SPMM_TMA ? fns().tn[kq] : fns().tw[kq]);
    p->smem = tma_smem_bytes(kq);
    GP_CHECK(encode_p_map(p->tmap, (const float*)c->P.p, c->n_act, kp));
  }
  GP_CUDA(cudaFuncSetAttribute(p->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem));
  int per_sm = 0;
  GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->fn, kSpmmThreads, p->smem));
  if (per_sm < 1) per_sm = 1;
  int64_t g = (c->nblk + kSpmmWarps - 1) / kSpmmWarps;
  if (g < 1) g = 1;
  if (g > (int64_t)c->num_sms * per_sm) g = (int64_t)c->num_sms * per_sm;
  p->grid = (unsigned)g;
  return GP_OK;
}

void spmm_launch(const SpmmPlan& p, cudaStream_t s, gp_ctx* c, CgState* st) {
  if (p.variant == GP_SPMM_WINDOW) {
    window_launch(p, s, c, st, p.k, p.m_hist);
    return;
  }
  int64_t n = c->n_act, nblk = c->nblk;
  const int64_t* brp = (const int64_t*)c->brp.p;
  const int32_t* bcol = (const int32_t*)c->bcol.p;
  const float4* bval = (const float4*)c->bval.p;
  const float4* P = (const float4*)c->P.p;
  float4* Q = (float4*)c->Q.p;
  double* part = (double*)c->part_a.p;
  if (p.variant == GP_SPMM_CPASYNC || p.variant == GP_SPMM_CPASYNC_WIDE) {
    Group g{nullptr, nullptr};
    void* args[] = {&n, &nblk, &brp, &bcol, &bval, &P, &Q, &part, &st, &g};
    cudaLaunchKernel(p.fn, dim3(p.grid), dim3(kSpmmThreads), args, p.smem, s);
  } else {
    void* args[] = {&n, &nblk, &brp, &bcol, &bval, (void*)p.tmap, &P, &Q, &part, &st};
    cudaLaunchKernel(p.fn, dim3(p.grid), dim3(kSpmmThreads), args, p.smem, s);
  }
}

void spmm_launch_io(const SpmmPlan& p, cudaStream_t s, gp_ctx* c, CgState* st, const float* in, float* out) {
  if (p.variant != GP_SPMM_CPASYNC && p.variant != GP_SPMM_CPASYNC_WIDE) return;
  int64_t n = c->n_act, nblk = c->nblk;
  const int64_t* brp = (const int64_t*)c->brp.p;
  const int32_t* bcol = (const int32_t*)c->bcol.p;
  const float4* bval = (const float4*)c->bval.p;
  const float4* P = (const float4*)in;
  float4* Q = (float4*)out;
  double* part = (double*)c->part_a.p;
  Group g{nullptr, nullptr};
  void* args[] = {&n, &nblk, &brp, &bcol, &bval, &P, &Q, &part, &st, &g};
  cudaLaunchKernel(p.fn, dim3(p.grid), dim3(kSpmmThreads), args, p.smem, s);
}

void spmm_launch_group(const SpmmPlan& p, cudaStream_t s, unsigned total, Group g) {
  if (p.variant != GP_SPMM_CPASYNC && p.variant != GP_SPMM_CPASYNC_WIDE) return;
  // every argument but the group is taken from the instance table
  int64_t n = 0, nblk = 0;
  const int64_t* brp = nullptr;
  const int32_t* bcol = nullptr;
  const float4* bval = nullptr;
  const float4* P = nullptr;
  float4* Q = nullptr;
  double* part = nullptr;
  CgState* st = nullptr;
  void* args[] = {&n, &nblk, &brp, &bcol, &bval, &P, &Q, &part, &st, &g};
  cudaLaunchKernel(p.fn, dim3(total), dim3(kSpmmThreads), args, p.smem, s);
}

int spmm_select(gp_ctx* c, int kp, int flags, CgState* st, SpmmPlan* plan, int k, int m_hist) {
  const int forced = (flags & GP_FLAG_SPMM_CPASYNC)        ? GP_SPMM_CPASYNC
                     : (flags & GP_FLAG_SPMM_TMA)          ? GP_SPMM_TMA
                     : (flags & GP_FLAG_SPMM_TMA_WIDE)     ? GP_SPMM_TMA_WIDE
                     : (flags & GP_FLAG_SPMM_CPASYNC_WIDE) ? GP_SPMM_CPASYNC_WIDE
                     : (flags & GP_FLAG_SPMM_WINDOW)       ? GP_SPMM_WINDOW
                                                           : -1;
  plan->k = k;
  plan->m_hist = m_hist;
  if (forced >= 0) {
    // a wide form that would hold one float4 per lane is its narrow form; the
    // window form needs the regrouped matrix
    int v = forced;
    if (v == GP_SPMM_WINDOW && !window_available(c, kp)) v = GP_SPMM_CPASYNC_WIDE;
    if (v != GP_SPMM_WINDOW && !spmm_available(v, kp))
      v = v == GP_SPMM_TMA_WIDE ? GP_SPMM_TMA : v == GP_SPMM_CPASYNC_WIDE ? GP_SPMM_CPASYNC : v;
    return spmm_plan(c, kp, v, plan);
  }
  const TuneKey key{c->device, kp, c->n_act, c->nblk, c->nbent};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto f = g_tuned.find(key);
    if (f != g_tuned.end()) {
      int v = f->second;
      if (v == GP_SPMM_WINDOW && !window_available(c, kp)) v = GP_SPMM_CPASYNC_WIDE;
      return spmm_plan(c, kp, v, plan);
    }
  }
  // time every available form on this matrix: one warm-up launch, then
  // three timed ones (the state is that of iteration 0, so the launches
  // compute Q = Khat P0 and the CG loop recomputes it)
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GP_CUDA(cudaEventCreate(&e0));
  GP_CUDA(cudaEventCreate(&e1));
  int best = GP_SPMM_CPASYNC;
  float best_ms = 0.f;
  int status = GP_OK;
  for (int v = GP_SPMM_CPASYNC; v <= GP_SPMM_WINDOW && status == GP_OK; ++v) {
    if (v == GP_SPMM_WINDOW ? !window_available(c, kp) : !spmm_available(v, kp)) continue;
    SpmmPlan p;
    p.k = k;
    p.m_hist = m_hist;
    status = spmm_plan(c, kp, v, &p);
    if (status != GP_OK) break;
    spmm_launch(p, c->stream, c, st);
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < 3; ++r) spmm_launch(p, c->stream, c, st);
    cudaEventRecord(e1, c->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      status = cuda_status(e);
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c->launches += 4;
    if (v == GP_SPMM_CPASYNC || ms < best_ms) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != GP_OK) return status;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto ins = g_tuned.emplace(key, best);  // a concurrent tuner's choice wins if it came first
    best = ins.first->second;
  }
  return spmm_plan(c, kp, best, plan);
}


}  // namespace gp
