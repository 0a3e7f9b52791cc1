// Q = Khat P through column windows (Sec. 2.5: the product of every CG
// iteration), the SpMM form GP_SPMM_WINDOW.
//
// The 8x1 block CSR (block row b = rows 8b..8b+7, Morton order) is regrouped
// once per assembly into tiles of kWT consecutive block rows.  The rows of a
// tile are close in space, so their blocks share columns: the sorted union of
// a tile's block columns (about 3.5 blocks per distinct column on the
// clustered 3-D workloads) is cut into segments of at most kWS columns and
// kWBcap blocks.  Per segment the assembly writes
//   * a record: kWT block counts (u16), each block's column as its position in
//     the segment (u8), and the blocks' 8 values (32 bytes each), grouped by
//     block row and ascending in column within a row;
//   * the segment's columns as runs of consecutive indices (start, length,
//     position), since neighbouring points are stored consecutively.
// The SpMM then runs one persistent CTA per SM over a contiguous range of
// tiles holding an equal share of the blocks: a producer warp streams the
// segments through a ring of shared-memory stages with the tensor-memory
// accelerator (one bulk copy per run of P rows, one for the record, all
// completing on the stage's mbarrier), and kWT consumer warps, one per block
// row of the tile, apply the segment's blocks to the staged rows of P.  Each
// row of P therefore crosses from L2 into shared memory once per tile instead
// of once per block, and no load/store-unit instruction stages data.  The
// last CTA to finish sums the CTAs' p^T q partials and forms the CG step
// alpha, so no separate reduction launch follows.
#include <climits>

#include "gp_internal.cuh"
#include "async.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBR = 8;                              // rows per block (8x1 blocks)
constexpr int kWT = 8;                              // block rows per tile = consumer warps
constexpr int kWS = 96;                             // columns per segment at most (fits u8)
constexpr int kWBcap = 384;                         // blocks per segment at most
constexpr int kWThreads = (kWT + 1) * 32;           // a consumer warp per block row, one producer
constexpr int kWRecMax = 16 + kWBcap + 32 * kWBcap; // record bytes at most
constexpr int kWRP = 2;                             // rows per pass of the epilogue sum
constexpr int kTileWarps = 4;                       // warps per CTA of the tiling builder

static_assert(kWBcap >= kWT, "a column can hit every block row of a tile");
static_assert(kWS <= 256, "positions in a segment are bytes");

// float4 columns per lane (as the wide cp.async form): a warp step applies
// NG = 32 / (KQ / LW) blocks
constexpr int win_lw(int kq) { return (kq % 3 == 0 && kq >= 6) ? 3 : (kq % 2 == 0 && kq >= 4) ? 2 : 1; }
constexpr int win_stage_bytes(int kq) { return (kWS * 16 * kq + kWRecMax + 127) / 128 * 128; }
constexpr int win_scratch_bytes(int kq) { return (32 / (kq / win_lw(kq))) * kWRP * kq * 16; }

__device__ inline int warp_min_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// ------------------------------------------------------------------ tiling
// One warp per tile; lane r < kWT walks the sorted column list of block row
// t kWT + r.  The warp merges the lists (warp minimum of the heads), so the
// union is visited in ascending order with each column's multiplicity; a new
// segment starts when the current one holds kWS columns or would exceed
// kWBcap blocks.  COUNT writes per tile the numbers of segments, runs and
// 16-byte record units; FILL writes descriptors, runs and records at the
// offsets the scans of those counts give.  Column lists are read through a
// 32-entry shared buffer per row so that the merge does not wait on a global
// load per step.
template <bool FILL>
__global__ void __launch_bounds__(kTileWarps * 32) k_wtile(int64_t nblk, int64_t ntiles,
                                                           const int64_t* __restrict__ brp,
                                                           const int32_t* __restrict__ bcol,
                                                           const float4* __restrict__ bval,
                                                           int32_t* __restrict__ t_nseg, int32_t* __restrict__ t_nrun,
                                                           int32_t* __restrict__ t_nrec,
                                                           const int64_t* __restrict__ tseg,
                                                           const int64_t* __restrict__ trun,
                                                           const int64_t* __restrict__ trec,
                                                           uint4* __restrict__ segd, int2* __restrict__ runs,
                                                           uint4* __restrict__ rec) {
  __shared__ int s_buf[kTileWarps][kWT][32];
  __shared__ uint8_t s_pos[kTileWarps][kWT][FILL ? kWBcap : 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t t = (int64_t)blockIdx.x * kTileWarps + w; t < ntiles; t += (int64_t)gridDim.x * kTileWarps) {
    int64_t pos = 0, end = 0;
    const int64_t b = t * kWT + lane;
    if (lane < kWT && b < nblk) {
      pos = brp[b];
      end = brp[b + 1];
    }
    int bi = 32;                 // next unread entry of this row's buffer (32: empty)
    int64_t seg_first = pos;     // this row's first block in the current segment
    int cnt = 0;                 // this row's blocks in the current segment
    // warp-uniform state
    int seg_ent = 0, seg_blk = 0, nseg = 0, nrun = 0, run_seg0 = 0;
    int64_t nrec = 0;
    int run_start = 0, run_len = 0, run_dst = 0, prev = -2;
    const int64_t seg_base = FILL ? tseg[t] : 0, run_base = FILL ? trun[t] : 0, rec_base = FILL ? trec[t] : 0;

    auto refill = [&]() {
      unsigned need = __ballot_sync(kFull, lane < kWT && bi == 32 && pos < end);
      while (need) {
        const int r = __ffs(need) - 1;
        need &= need - 1u;
        const int64_t p0 = __shfl_sync(kFull, pos, r), e0 = __shfl_sync(kFull, end, r);
        s_buf[w][r][lane] = p0 + lane < e0 ? bcol[p0 + lane] : INT_MAX;
        if (lane == r) bi = 0;
      }
      __syncwarp();
    };
    auto flush_run = [&]() {
      if (run_len > 0) {
        if (FILL && lane == 0) runs[run_base + nrun] = make_int2(run_start, run_len | (run_dst << 16));
        ++nrun;
        run_len = 0;
      }
    };
    auto close_seg = [&]() {
      if (seg_ent == 0) return;
      flush_run();
      const int nb = seg_blk;
      const int pad = (nb + 15) / 16 * 16;
      const int64_t units = 1 + pad / 16 + 2 * nb;
      if (FILL) {
        // exclusive prefix of the rows' counts, known to every lane
        int off[kWT];
        int64_t first[kWT];
        int acc = 0;
#pragma unroll
        for (int r = 0; r < kWT; ++r) {
          off[r] = acc;
          acc += __shfl_sync(kFull, cnt, r);
          first[r] = __shfl_sync(kFull, seg_first, r);
        }
        unsigned char* base = (unsigned char*)(rec + rec_base + nrec);
        if (lane < kWT) ((uint16_t*)base)[lane] = (uint16_t)cnt;
        for (int q = nb + lane; q < pad; q += 32) base[16 + q] = 0;
        float4* dv = (float4*)(base + 16 + pad);
        for (int q = lane; q < nb; q += 32) {
          int r = 0;
#pragma unroll
          for (int rr = 1; rr < kWT; ++rr)
            if (off[rr] <= q) r = rr;
          const int kk = q - off[r];
          const int64_t src = first[r] + kk;
          base[16 + q] = s_pos[w][r][kk];
          dv[2 * q] = bval[2 * src];
          dv[2 * q + 1] = bval[2 * src + 1];
        }
        if (lane == 0)
          segd[seg_base + nseg] = make_uint4((unsigned)(rec_base + nrec), (unsigned)units,
                                             (unsigned)(run_base + run_seg0),
                                             (unsigned)(nrun - run_seg0) | ((unsigned)seg_ent << 16));
      }
      nrec += units;
      ++nseg;
      seg_ent = 0;
      seg_blk = 0;
      cnt = 0;
      seg_first = pos;
      run_seg0 = nrun;
      prev = -2;
      __syncwarp();
    };

    refill();
    for (;;) {
      const int hd = (lane < kWT && pos < end) ? s_buf[w][lane][bi] : INT_MAX;
      const int m = warp_min_int(hd);
      if (m == INT_MAX) break;
      const bool mine = hd == m;
      const int mult = __popc(__ballot_sync(kFull, mine));
      if (seg_ent == kWS || seg_blk + mult > kWBcap) close_seg();
      if (!(run_len > 0 && m == prev + 1)) {
        flush_run();
        run_start = m;
        run_dst = seg_ent;
      }
      ++run_len;
      prev = m;
      if (mine) {
        if (FILL) s_pos[w][lane][cnt] = (uint8_t)seg_ent;
        ++cnt;
        ++pos;
        ++bi;
      }
      ++seg_ent;
      seg_blk += mult;
      refill();
    }
    close_seg();
    if (!FILL && lane == 0) {
      t_nseg[t] = nseg;
      t_nrun[t] = nrun;
      t_nrec[t] = (int32_t)nrec;
    }
  }
}

// ------------------------------------------------------------------ SpMM
// first tile whose first block (brp at block row t kWT) is >= target
__device__ inline int64_t first_tile_at_or_after(const int64_t* __restrict__ brp, int64_t nblk, int64_t ntiles,
                                                  int64_t target) {
  int64_t lo = 0, hi = ntiles;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int64_t b = mid * kWT < nblk ? mid * kWT : nblk;
    if (__ldg(brp + b) < target) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Bounded wait that also gives up when another warp of the CTA gave up.
__device__ inline bool win_wait(uint64_t* b, unsigned parity, volatile int* abort_flag) {
  if (mbar_test(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(b, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

// The producer's part, run by lanes of warp 0: issue segment `sg` (its
// descriptor d and runs rc, lane l holding runs l, l + 32, l + 64) into
// stage s.  False if a descriptor would copy outside P or the stage: nothing
// is issued then and the caller stops the product.
template <int KQ>
__device__ inline bool win_issue(const uint4& d, const int2 (&rc)[3], int64_t n, int64_t nrun_total,
                                 unsigned char* stage, uint64_t* full, const uint4* __restrict__ rec,
                                 const float4* __restrict__ P) {
  constexpr int ROWB = 16 * KQ;
  const int lane = threadIdx.x & 31;
  const int nr = (int)(d.w & 0xffffu);
  int rows = 0;
  bool bad = nr > kWS || d.y == 0 || d.y * 16u > (unsigned)kWRecMax || (int64_t)d.z + nr > nrun_total;
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    if (lane + 32 * u < nr) {
      const int len = rc[u].y & 0xffff, dst = (rc[u].y >> 16) & 0xffff;
      bad = bad || rc[u].x < 0 || len < 1 || (int64_t)rc[u].x + len > n || dst + len > kWS;
      rows += len;
    }
  }
  if (__any_sync(kFull, bad)) return false;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rows += __shfl_xor_sync(kFull, rows, o);
  if (lane == 0) {
    mbar_arrive_expect(full, d.y * 16u + (unsigned)rows * ROWB);
    bulk_to_smem(stage + kWS * ROWB, rec + d.x, d.y * 16u, full);
  }
  __syncwarp();
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    if (lane + 32 * u < nr) {
      const int len = rc[u].y & 0xffff, dst = (rc[u].y >> 16) & 0xffff;
      bulk_to_smem(stage + dst * ROWB, P + (int64_t)rc[u].x * KQ, (unsigned)len * ROWB, full);
    }
  }
  return true;
}

// Descriptor of segment sg and a superset of its runs (the runs of
// consecutive segments are stored one after the other, so the loads need not
// wait for the descriptor).
__device__ inline void win_fetch(int64_t sg, int64_t s1, int64_t run0, const uint4* __restrict__ segd,
                                 const int2* __restrict__ runs, int64_t nrun_total, uint4& d, int2 (&rc)[3]) {
  const int lane = threadIdx.x & 31;
  d = sg < s1 ? segd[sg] : make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int64_t r = run0 + lane + 32 * u;
    rc[u] = sg < s1 && r < nrun_total ? runs[r] : make_int2(0, 0);
  }
}

template <int KQ, int LW>
__global__ void __launch_bounds__(kWThreads, 1) k_wspmm(int64_t n, int64_t nblk, int64_t ntiles,
                                                        const int64_t* __restrict__ brp,
                                                        const int64_t* __restrict__ tseg,
                                                        const uint4* __restrict__ segd,
                                                        const int2* __restrict__ runs,
                                                        const uint4* __restrict__ rec,
                                                        const float4* __restrict__ P, float4* __restrict__ Q,
                                                        double* __restrict__ part, gp::CgState* st, int k,
                                                        double* hist_alpha, int m_hist, int ns,
                                                        int64_t nrun_total) {
  const int it = st->iter;
  if (st->fin[it & 1]) return;
  static_assert(KQ % LW == 0, "LW must divide KQ");
  static_assert(kWS <= 96, "three runs per producer lane");
  constexpr int G = KQ / LW;   // lanes per block
  constexpr int NG = 32 / G;   // blocks per warp step
  constexpr int KP = 4 * KQ;
  constexpr int SB = win_stage_bytes(KQ);
  constexpr int SCR = win_scratch_bytes(KQ);
  constexpr int M = 32 / KQ;   // rows summed at once in the epilogue
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  uint64_t* full = (uint64_t*)(base + (size_t)ns * SB + (size_t)kWT * SCR);
  uint64_t* empty = full + ns;
  __shared__ int s_abort;
  __shared__ double shp[kWT][32][4];
  __shared__ double red[kWThreads];
  __shared__ double pq_sum[gp::kMaxCols];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kWT);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  const int64_t total = brp[nblk];
  const int64_t t0 = first_tile_at_or_after(brp, nblk, ntiles, total * blockIdx.x / gridDim.x);
  const int64_t t1 = first_tile_at_or_after(brp, nblk, ntiles, total * (blockIdx.x + 1) / gridDim.x);
  const int64_t s0 = tseg[t0], s1 = tseg[t1];  // this CTA's segments, in order

  gpd::Dot2 pq0, pq1, pq2, pq3;
  const int slot = lane < M * KQ ? lane % KQ : -1;
  if (w == kWT) {
    // ---------------- producer warp: segment i of the CTA into stage i % ns;
    // the next segment's descriptor and runs load while the current one
    // waits for its stage
    uint4 d;
    int2 rc[3];
    win_fetch(s0, s1, s0 < s1 ? (int64_t)segd[s0].z : 0, segd, runs, nrun_total, d, rc);
    int64_t i = 0;
    for (int64_t sg = s0; sg < s1; ++sg, ++i) {
      uint4 dn;
      int2 rn[3];
      win_fetch(sg + 1, s1, (int64_t)d.z + (d.w & 0xffffu), segd, runs, nrun_total, dn, rn);
      const int s = (int)(i % ns);
      if (i >= ns && !win_wait(&empty[s], (unsigned)(((i / ns) - 1) & 1), &s_abort)) break;
      if (!win_issue<KQ>(d, rc, n, nrun_total, base + (size_t)s * SB, &full[s], rec, P)) {
        if (lane == 0) {
          s_abort = 1;
          st->status = GP_ERR_CUDA;
        }
        break;
      }
      d = dn;
#pragma unroll
      for (int u = 0; u < 3; ++u) rc[u] = rn[u];
    }
    if (s_abort) {
      // leave no copy in flight: wait (bounded) for the stages issued last
      for (int64_t j = i > ns ? i - ns : 0; j < i; ++j)
        if (lane == 0) mbar_wait(&full[j % ns], (unsigned)((j / ns) & 1));
      __syncwarp();
    }
  } else {
    // ---------------- consumers: warp w applies block row t kWT + w
    const int grp = lane / G, gl = lane - grp * G;
    const bool act = grp < NG;
    float2 acc[kBR][2 * LW];
#pragma unroll
    for (int r = 0; r < kBR; ++r)
#pragma unroll
      for (int u = 0; u < 2 * LW; ++u) acc[r][u] = make_float2(0.f, 0.f);
    float4* scr = (float4*)(base + (size_t)ns * SB + (size_t)w * SCR);
    int64_t i = 0;
    bool ok = true;
    for (int64_t t = t0; t < t1 && ok; ++t) {
      const int64_t te = tseg[t + 1];
      for (int64_t sg = tseg[t]; sg < te; ++sg, ++i) {
        const int s = (int)(i % ns);
        if (!win_wait(&full[s], (unsigned)((i / ns) & 1), &s_abort)) {
          ok = false;
          break;
        }
        const unsigned char* stage = base + (size_t)s * SB;
        const unsigned char* recp = stage + kWS * 16 * KQ;
        const uint4 hdr = *(const uint4*)recp;
        const unsigned cw[4] = {hdr.x, hdr.y, hdr.z, hdr.w};
        int off = 0, nb = 0, mine = 0;
#pragma unroll
        for (int r = 0; r < kWT; ++r) {
          const int c = (int)((cw[r >> 1] >> (16 * (r & 1))) & 0xffffu);
          if (r < w) off += c;
          if (r == w) mine = c;
          nb += c;
        }
        const uint8_t* idxp = recp + 16;
        const float* vals = (const float*)(recp + 16 + (nb + 15) / 16 * 16);
        const float* Ps = (const float*)stage;
        for (int t2 = 0; t2 < mine; t2 += NG) {
          const int q = t2 + grp;
          if (act && q < mine) {
            const int kk = off + q;
            const float* prow = Ps + (int)idxp[kk] * KP + 4 * LW * gl;
            float4 pj[LW];
#pragma unroll
            for (int u = 0; u < LW; ++u) pj[u] = *(const float4*)(prow + 4 * u);
            const float4 v0 = *(const float4*)(vals + kk * kBR);
            const float4 v1 = *(const float4*)(vals + kk * kBR + 4);
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
        if (lane == 0) mbar_arrive(&empty[s]);
      }
      if (!ok) break;
      // the tile is done: the groups' partial rows of block row b are added
      // through the warp's scratch, kWRP rows per pass; the rows of P for
      // p^T q are loaded first, all passes at once
      const int64_t b = t * kWT + w;
      float4 pp[kBR / kWRP][kWRP];
#pragma unroll
      for (int r0 = 0; r0 < kBR; r0 += kWRP)
#pragma unroll
        for (int j = 0; j < kWRP; ++j) {
          const int r = lane / KQ + M * j;
          const int64_t row = b * kBR + r0 + r;
          pp[r0 / kWRP][j] = slot >= 0 && b < nblk && r < kWRP && row < n ? __ldg(P + row * KQ + slot)
                                                                           : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int r0 = 0; r0 < kBR; r0 += kWRP) {
        if (act) {
#pragma unroll
          for (int r = 0; r < kWRP; ++r)
#pragma unroll
            for (int u = 0; u < LW; ++u)
              scr[(grp * kWRP + r) * KQ + gl * LW + u] = make_float4(
                  acc[r0 + r][2 * u].x, acc[r0 + r][2 * u].y, acc[r0 + r][2 * u + 1].x, acc[r0 + r][2 * u + 1].y);
        }
        __syncwarp();
        if (slot >= 0 && b < nblk) {
#pragma unroll
          for (int j = 0; j < kWRP; ++j) {
            const int r = lane / KQ + M * j;
            if (r >= kWRP) break;
            float4 sum = scr[r * KQ + slot];
            for (int g2 = 1; g2 < NG; ++g2) {
              const float4 v = scr[(g2 * kWRP + r) * KQ + slot];
              sum.x += v.x;
              sum.y += v.y;
              sum.z += v.z;
              sum.w += v.w;
            }
            const int64_t row = b * kBR + r0 + r;
            if (row < n) {
              Q[row * KQ + slot] = sum;
              const float4 pv = pp[r0 / kWRP][j];
              pq0.add(pv.x, sum.x);
              pq1.add(pv.y, sum.y);
              pq2.add(pv.z, sum.z);
              pq3.add(pv.w, sum.w);
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
    shp[w][lane][0] = slot >= 0 ? pq0.value() : 0.0;
    shp[w][lane][1] = slot >= 0 ? pq1.value() : 0.0;
    shp[w][lane][2] = slot >= 0 ? pq2.value() : 0.0;
    shp[w][lane][3] = slot >= 0 ? pq3.value() : 0.0;
  }
  __syncthreads();
  if (s_abort && threadIdx.x == 0 && st->status == GP_OK) st->status = GP_ERR_TIMEOUT;
  // this CTA's p^T q partials, in a fixed order
  if (threadIdx.x < KP) {
    const int qq = threadIdx.x >> 2, cc = threadIdx.x & 3;
    double tsum = 0.0;
    for (int ww = 0; ww < kWT; ++ww)
      for (int l = 0; l < 32; ++l)
        if ((l < M * KQ ? l % KQ : -1) == qq) tsum += shp[ww][l][cc];
    part[(int64_t)blockIdx.x * KP + threadIdx.x] = tsum;
  }
  // the last CTA to finish forms alpha from all partials
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicInc(&st->ticket_a, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  gpd::block_sum_partials(part, (int)gridDim.x, KP, KP, pq_sum, red);
  gpd::cg_alpha_finish(st, it, pq_sum, k, KP, hist_alpha, m_hist);
}

typedef void (*WinFn)(int64_t, int64_t, int64_t, const int64_t*, const int64_t*, const uint4*, const int2*,
                      const uint4*, const float4*, float4*, double*, gp::CgState*, int, double*, int, int, int64_t);

template <int KQ>
void fill_win(WinFn* f) {
  f[KQ] = k_wspmm<KQ, win_lw(KQ)>;
}

struct WinTable {
  WinFn f[18] = {};
  WinTable() {
    fill_win<1>(f);
    fill_win<2>(f);
    fill_win<3>(f);
    fill_win<4>(f);
    fill_win<5>(f);
    fill_win<6>(f);
    fill_win<7>(f);
    fill_win<8>(f);
    fill_win<9>(f);
    fill_win<10>(f);
    fill_win<11>(f);
    fill_win<12>(f);
    fill_win<13>(f);
    fill_win<14>(f);
    fill_win<15>(f);
    fill_win<16>(f);
    fill_win<17>(f);
  }
};
const WinTable& win_fns() {
  static const WinTable t;
  return t;
}

unsigned grid_for(int64_t items, int per_block, int max_blocks) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (unsigned)g;
}

int read_i64(gp_ctx* c, const int64_t* dev, int64_t* out) {
  GP_CHECK(gp::ensure_pinned(c, sizeof(int64_t)));
  GP_CUDA(cudaMemcpyAsync(c->pinned, dev, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  GP_CUDA(cudaStreamSynchronize(c->stream));
  *out = *(int64_t*)c->pinned;
  return GP_OK;
}

}  // namespace

namespace gp {

int window_build(gp_ctx* c) {
  c->w_ntiles = 0;
  c->w_nseg = 0;
  const int64_t nblk = c->nblk;
  if (nblk == 0) return GP_OK;
  const int64_t ntiles = (nblk + kWT - 1) / kWT;
  if (ntiles > ((int64_t)1 << 30)) return GP_ERR_UNSUPPORTED;
  GP_CHECK(ensure(c, c->w_cnt, (size_t)ntiles * 3 * sizeof(int32_t)));
  GP_CHECK(ensure(c, c->w_tseg, (size_t)(ntiles + 1) * sizeof(int64_t)));
  GP_CHECK(ensure(c, c->w_trun, (size_t)(ntiles + 1) * sizeof(int64_t)));
  GP_CHECK(ensure(c, c->w_trec, (size_t)(ntiles + 1) * sizeof(int64_t)));
  int32_t* cnt = (int32_t*)c->w_cnt.p;
  const unsigned g = grid_for(ntiles, kTileWarps, c->num_sms * 16);
  k_wtile<false><<<g, kTileWarps * 32, 0, c->stream>>>(nblk, ntiles, (const int64_t*)c->brp.p,
                                                       (const int32_t*)c->bcol.p, (const float4*)c->bval.p, cnt,
                                                       cnt + ntiles, cnt + 2 * ntiles, nullptr, nullptr, nullptr,
                                                       nullptr, nullptr, nullptr);
  GP_LAUNCH_CHECK();
  c->launches += 1;
  GP_CHECK(scan_i32_to_i64(c, cnt, (int64_t*)c->w_tseg.p, ntiles));
  GP_CHECK(scan_i32_to_i64(c, cnt + ntiles, (int64_t*)c->w_trun.p, ntiles));
  GP_CHECK(scan_i32_to_i64(c, cnt + 2 * ntiles, (int64_t*)c->w_trec.p, ntiles));
  int64_t nseg = 0, nrun = 0, nrec = 0;
  GP_CHECK(read_i64(c, (const int64_t*)c->w_tseg.p + ntiles, &nseg));
  GP_CHECK(read_i64(c, (const int64_t*)c->w_trun.p + ntiles, &nrun));
  GP_CHECK(read_i64(c, (const int64_t*)c->w_trec.p + ntiles, &nrec));
  // descriptors hold run and record offsets as 32-bit numbers
  if (nrun >= ((int64_t)1 << 32) || nrec >= ((int64_t)1 << 32)) return GP_ERR_UNSUPPORTED;
  GP_CHECK(ensure(c, c->w_segd, (size_t)nseg * sizeof(uint4)));
  GP_CHECK(ensure(c, c->w_runs, (size_t)nrun * sizeof(int2)));
  GP_CHECK(ensure(c, c->w_rec, (size_t)nrec * 16));
  k_wtile<true><<<g, kTileWarps * 32, 0, c->stream>>>(nblk, ntiles, (const int64_t*)c->brp.p,
                                                      (const int32_t*)c->bcol.p, (const float4*)c->bval.p, nullptr,
                                                      nullptr, nullptr, (const int64_t*)c->w_tseg.p,
                                                      (const int64_t*)c->w_trun.p, (const int64_t*)c->w_trec.p,
                                                      (uint4*)c->w_segd.p, (int2*)c->w_runs.p, (uint4*)c->w_rec.p);
  GP_LAUNCH_CHECK();
  c->launches += 1;
  c->w_ntiles = ntiles;
  c->w_nseg = nseg;
  c->w_nrun = nrun;
  return GP_OK;
}

bool window_available(gp_ctx* c, int kp) {
  if (kp % 4 || kp < 4 || kp > 4 * 17) return false;
  return c->nblk > 0 && c->precision == GP_FP32_MIXED && win_fns().f[kp / 4] != nullptr;
}

int window_plan(gp_ctx* c, int kp, SpmmPlan* p) {
  if (!window_available(c, kp)) return GP_ERR_UNSUPPORTED;
  // the regrouped matrix of this assembly, built on first use
  if (c->w_ntiles == 0) GP_CHECK(window_build(c));
  const int kq = kp / 4;
  int smem_max = 0;
  GP_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  // static shared memory of the kernel: partial sums and flags
  const size_t fixed = sizeof(double) * (kWT * 32 * 4 + kWThreads + gp::kMaxCols) + 64;
  const size_t scr = (size_t)kWT * win_scratch_bytes(kq);
  const size_t sb = win_stage_bytes(kq);
  int ns = 8;
  while (ns > 2 && 128 + ns * sb + scr + 16 * ns + fixed > (size_t)smem_max) --ns;
  if (128 + ns * sb + scr + 16 * ns + fixed > (size_t)smem_max) return GP_ERR_UNSUPPORTED;
  p->variant = GP_SPMM_WINDOW;
  p->kp = kp;
  p->fn = (const void*)win_fns().f[kq];
  p->smem = 128 + ns * sb + scr + 16 * ns;
  p->stages = ns;
  p->fused_alpha = true;
  GP_CUDA(cudaFuncSetAttribute(p->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem));
  int per_sm = 0;
  GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->fn, kWThreads, p->smem));
  if (per_sm < 1) return GP_ERR_UNSUPPORTED;
  int64_t gsz = c->w_ntiles < (int64_t)c->num_sms ? c->w_ntiles : (int64_t)c->num_sms;
  p->grid = (unsigned)(gsz < 1 ? 1 : gsz);
  return GP_OK;
}

void window_launch(const SpmmPlan& p, cudaStream_t s, gp_ctx* c, CgState* st, int k, int m_hist) {
  int64_t n = c->n_act, nblk = c->nblk, ntiles = c->w_ntiles;
  const int64_t* brp = (const int64_t*)c->brp.p;
  const int64_t* tseg = (const int64_t*)c->w_tseg.p;
  const uint4* segd = (const uint4*)c->w_segd.p;
  const int2* runs = (const int2*)c->w_runs.p;
  const uint4* rec = (const uint4*)c->w_rec.p;
  const float4* P = (const float4*)c->P.p;
  float4* Q = (float4*)c->Q.p;
  double* part = (double*)c->part_a.p;
  double* ha = (double*)c->hist_alpha.p;
  int ns = p.stages;
  int64_t nrun = c->w_nrun;
  void* args[] = {&n, &nblk, &ntiles, &brp, &tseg, &segd, &runs, &rec, &P, &Q, &part, &st, &k, &ha, &m_hist, &ns,
                  &nrun};
  cudaLaunchKernel(p.fn, dim3(p.grid), dim3(kWThreads), args, p.smem, s);
}

}  // namespace gp
