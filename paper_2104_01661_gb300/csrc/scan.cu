// Graph-store primitives: exclusive scan, stable radix sort, stable compaction of heavy rows and
// the CSR -> CSC transpose (Property_AT, Sec. II-A).  All deterministic.
#include <algorithm>
#include <iterator>
#include <vector>

#include "internal.cuh"

namespace lagr {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void scan_tile_sums(const int32_t *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
  __shared__ int64_t red[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t s = 0;
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
    const int64_t k = base + i;
    if (k < n) s += in[k];
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) sums[blockIdx.x] = s;
}

// exclusive scan of the tile sums, in place, by one block of 1024 threads
__global__ void scan_tile_offsets(int64_t *__restrict__ sums, int64_t ntiles, int32_t *__restrict__ out_total,
                                  int64_t n) {
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < ntiles; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = (i < ntiles) ? sums[i] : 0;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(LAGR_FULL_MASK, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t w = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(LAGR_FULL_MASK, w, o);
        if (lane >= o) w += t;
      }
      warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int64_t before = carry + (warp > 0 ? warp_tot[warp - 1] : 0);
    if (i < ntiles) sums[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) out_total[n] = (int32_t)carry;
}

__global__ void scan_tile_apply(const int32_t *__restrict__ in, int64_t n, const int64_t *__restrict__ offs,
                                int32_t *__restrict__ out) {
  __shared__ int64_t warp_tot[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int32_t v[SCAN_ITEMS];
  int64_t tsum = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; j++) {
    const int64_t k = base + j;
    v[j] = (k < n) ? in[k] : 0;
    tsum += v[j];
  }
  int64_t x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(LAGR_FULL_MASK, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  int64_t before = offs[blockIdx.x];
  for (int w = 0; w < warp; w++) before += warp_tot[w];
  int64_t run = before + x - tsum;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; j++) {
    const int64_t k = base + j;
    if (k < n) out[k] = (int32_t)run;
    run += v[j];
  }
}

// ---- radix sort ------------------------------------------------------------------------------

constexpr int RADIX_THREADS = 256;
constexpr int RADIX_ROUNDS = 16;
constexpr int RADIX_TILE = RADIX_THREADS * RADIX_ROUNDS;
constexpr int RADIX_BINS = 256;

__global__ void radix_hist(const int32_t *__restrict__ keys, int64_t n, int shift, int32_t *__restrict__ hist,
                           int nblocks) {
  __shared__ int32_t h[RADIX_BINS];
  for (int i = threadIdx.x; i < RADIX_BINS; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RADIX_TILE;
  for (int i = threadIdx.x; i < RADIX_TILE; i += blockDim.x) {
    const int64_t k = base + i;
    if (k < n) atomicAdd(&h[((uint32_t)keys[k] >> shift) & (RADIX_BINS - 1)], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RADIX_BINS; d += blockDim.x) hist[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

// stable scatter: keys of this tile go, in index order within each digit, to offs[digit][block]
__global__ void radix_scatter(const int32_t *__restrict__ keys, const int32_t *__restrict__ vals, int64_t n,
                              int shift, const int32_t *__restrict__ offs, int nblocks,
                              int32_t *__restrict__ keys_out, int32_t *__restrict__ vals_out) {
  __shared__ int32_t running[RADIX_BINS];
  __shared__ int32_t wcnt[RADIX_THREADS / 32][RADIX_BINS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < RADIX_BINS; d += blockDim.x) running[d] = offs[(int64_t)d * nblocks + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * RADIX_TILE;
  for (int r = 0; r < RADIX_ROUNDS; r++) {
    for (int i = threadIdx.x; i < (RADIX_THREADS / 32) * RADIX_BINS; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t idx = base + (int64_t)r * RADIX_THREADS + threadIdx.x;
    const bool valid = idx < n;
    const int32_t key = valid ? keys[idx] : 0;
    const int digit = ((uint32_t)key >> shift) & (RADIX_BINS - 1);
    const unsigned peers = __match_any_sync(LAGR_FULL_MASK, valid ? digit : (RADIX_BINS + 1));
    const int rank_in_warp = __popc(peers & lanemask_lt());
    const bool leader = (__ffs(peers) - 1) == lane;
    if (valid && leader) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    if (valid) {
      int32_t pos = running[digit] + rank_in_warp;
      for (int w = 0; w < warp; w++) pos += wcnt[w][digit];
      keys_out[pos] = key;
      vals_out[pos] = vals[idx];
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX_BINS; d += blockDim.x) {
      int32_t add = 0;
#pragma unroll
      for (int w = 0; w < RADIX_THREADS / 32; w++) add += wcnt[w][d];
      running[d] += add;
    }
    __syncthreads();
  }
}

// ---- heavy-row compaction ---------------------------------------------------------------------

__global__ void scatter_heavy(const int32_t *__restrict__ flag, const int32_t *__restrict__ pos, int32_t n,
                              int32_t *__restrict__ list) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) list[pos[i]] = (int32_t)i;
}

// ---- transpose ------------------------------------------------------------------------------

__global__ void iota_kernel(int32_t *__restrict__ a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

// row id of every stored entry: one warp per row
__global__ void expand_rows(const int32_t *__restrict__ rowptr, int32_t n, int32_t *__restrict__ rowid) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int32_t b = rowptr[i], e = rowptr[i + 1];
    for (int32_t k = b + lane; k < e; k += 32) rowid[k] = (int32_t)i;
  }
}

__global__ void count_cols(const int32_t *__restrict__ colidx, int64_t nnz, int32_t *__restrict__ cnt) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[colidx[k]], 1);
}

__global__ void gather_transpose(const int32_t *__restrict__ perm, const int32_t *__restrict__ rowid,
                                 const float *__restrict__ val, int64_t nnz, int32_t *__restrict__ at_colidx,
                                 float *__restrict__ at_val) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = perm[k];
    at_colidx[k] = rowid[e];
    if (at_val) at_val[k] = val[e];
  }
}

// ---- row plan -----------------------------------------------------------------------------------

// per row: 1 if it is heavy (more than `heavy` entries), and its light degree (0 for a heavy row)
__global__ void row_classes(const int32_t *__restrict__ rowptr, int32_t n, int32_t heavy, int32_t *__restrict__ hflag,
                            int32_t *__restrict__ ld) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = rowptr[i + 1] - rowptr[i];
    hflag[i] = d > heavy;
    ld[i] = d <= heavy ? d : 0;
  }
}

// every block start: the rows b0[0 .. nb0-1] (below n), each heavy row and the row after it
__global__ void mark_cuts(const int32_t *__restrict__ b0, int32_t nb0, const int32_t *__restrict__ heavy, int32_t nh,
                          int32_t n, int32_t *__restrict__ mark) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb0; i += stride)
    if (b0[i] < n) mark[b0[i]] = 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nh; i += stride) {
    mark[heavy[i]] = 1;
    if (heavy[i] + 1 < n) mark[heavy[i] + 1] = 1;
  }
}

// the marked rows in order become blk[]; a block that starts at a heavy row is that row alone
__global__ void scatter_blocks(const int32_t *__restrict__ mark, const int32_t *__restrict__ mpos,
                               const int32_t *__restrict__ rowptr, int32_t n, int32_t heavy,
                               int32_t *__restrict__ blk, uint8_t *__restrict__ hblk) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride)
    if (mark[r]) {
      blk[mpos[r]] = (int32_t)r;
      hblk[mpos[r]] = (rowptr[r + 1] - rowptr[r]) > heavy;
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n == 0) {  // one empty block
      blk[0] = 0;
      blk[1] = 0;
      hblk[0] = 0;
    } else {
      blk[mpos[n]] = n;
    }
  }
}

// blk[b] = first row r with lp[r] + r >= b * units (lp = exclusive prefix of light degrees)
__global__ void block_starts(const int32_t *__restrict__ lp, int32_t n, int32_t nblk, int32_t units,
                             int32_t *__restrict__ blk) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= nblk; b += (int64_t)gridDim.x * blockDim.x) {
    if (b == nblk) {
      blk[b] = n;
      continue;
    }
    const int64_t target = b * (int64_t)units;
    int32_t lo = 0, hi = n;  // answer in [lo, hi]
    while (lo < hi) {
      const int32_t mid = lo + ((hi - lo) >> 1);
      if ((int64_t)lp[mid] + mid >= target) hi = mid; else lo = mid + 1;
    }
    blk[b] = lo;
  }
}

__global__ void heavy_chunk_counts(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ heavy, int32_t nh,
                                   int32_t hchunk, int32_t *__restrict__ nch) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = rowptr[heavy[h] + 1] - rowptr[heavy[h]];
    nch[h] = (d + hchunk - 1) / hchunk;
  }
}

__global__ void heavy_chunk_rows(const int32_t *__restrict__ hc_off, int32_t nh, int32_t *__restrict__ hc_row) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += (int64_t)gridDim.x * blockDim.x)
    for (int32_t c = hc_off[h]; c < hc_off[h + 1]; c++) hc_row[c] = (int32_t)h;
}

}  // namespace

int64_t scan_scratch_len(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

int exclusive_scan(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s, char *msg, int64_t *scratch) {
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (ntiles == 0) {
    LAGR_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
    return LAGR_OK;
  }
  Temp<int64_t> sums(s);
  int64_t *sp = scratch;
  if (!sp) {
    LAGR_TRY(sums.alloc(ntiles, msg, "scan tile sums"));
    sp = sums.p;
  }
  scan_tile_sums<<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(in, n, sp);
  scan_tile_offsets<<<1, 1024, 0, s>>>(sp, ntiles, out, n);
  scan_tile_apply<<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(in, n, sp, out);
  LAGR_LAUNCH_CHECK();
  return LAGR_OK;
}

int64_t radix_scratch_len(int64_t n) {
  const int64_t nblocks = (n + RADIX_TILE - 1) / RADIX_TILE;
  return 2 * (nblocks * RADIX_BINS + 1);
}

int radix_sort_pairs(int32_t *keys, int32_t *vals, int32_t *tmp_k, int32_t *tmp_v, int64_t n, int bits,
                     cudaStream_t s, char *msg, int32_t *scratch, int64_t *scan_scratch) {
  if (n <= 1) return LAGR_OK;
  const int64_t nblocks = (n + RADIX_TILE - 1) / RADIX_TILE;
  Temp<int32_t> own(s);
  int32_t *hist = scratch;
  if (!hist) {
    LAGR_TRY(own.alloc(radix_scratch_len(n), msg, "radix histogram"));
    hist = own.p;
  }
  int32_t *offs = hist + nblocks * RADIX_BINS + 1;
  int32_t *k_in = keys, *v_in = vals, *k_out = tmp_k, *v_out = tmp_v;
  int passes = 0;
  for (int shift = 0; shift < bits; shift += 8, passes++) {
    radix_hist<<<(unsigned)nblocks, RADIX_THREADS, 0, s>>>(k_in, n, shift, hist, (int)nblocks);
    LAGR_TRY(exclusive_scan(hist, offs, nblocks * RADIX_BINS, s, msg, scan_scratch));
    radix_scatter<<<(unsigned)nblocks, RADIX_THREADS, 0, s>>>(k_in, v_in, n, shift, offs, (int)nblocks, k_out,
                                                             v_out);
    LAGR_LAUNCH_CHECK();
    int32_t *t = k_in; k_in = k_out; k_out = t;
    t = v_in; v_in = v_out; v_out = t;
  }
  if (passes & 1) {
    LAGR_CUDA_TRY(cudaMemcpyAsync(keys, k_in, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    LAGR_CUDA_TRY(cudaMemcpyAsync(vals, v_in, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
  return LAGR_OK;
}

int transpose_csr(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *colidx, const float *val,
                  int32_t *at_rowptr, int32_t *at_colidx, float *at_val, cudaStream_t s, char *msg) {
  Temp<int32_t> cnt(s);
  LAGR_TRY(cnt.alloc((size_t)n + 1, msg, "transpose counts"));
  LAGR_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, ((size_t)n + 1) * sizeof(int32_t), s));
  if (nnz > 0) count_cols<<<grid_for(nnz, 256), 256, 0, s>>>(colidx, nnz, cnt.p);
  LAGR_LAUNCH_CHECK();
  LAGR_TRY(exclusive_scan(cnt.p, at_rowptr, n, s, msg));
  if (nnz == 0) return LAGR_OK;
  Temp<int32_t> keys(s), perm(s), tk(s), tv(s), rowid(s);
  LAGR_TRY(keys.alloc(nnz, msg, "transpose keys"));
  LAGR_TRY(perm.alloc(nnz, msg, "transpose permutation"));
  LAGR_TRY(tk.alloc(nnz, msg, "transpose work"));
  LAGR_TRY(tv.alloc(nnz, msg, "transpose work"));
  LAGR_TRY(rowid.alloc(nnz, msg, "transpose row ids"));
  LAGR_CUDA_TRY(cudaMemcpyAsync(keys.p, colidx, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  iota_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(perm.p, nnz);
  expand_rows<<<grid_for((int64_t)n * 32, 256), 256, 0, s>>>(rowptr, n, rowid.p);
  LAGR_LAUNCH_CHECK();
  int bits = 1;
  while (bits < 31 && ((int64_t)1 << bits) < (int64_t)n) bits++;
  LAGR_TRY(radix_sort_pairs(keys.p, perm.p, tk.p, tv.p, nnz, bits, s, msg));
  gather_transpose<<<grid_for(nnz, 256), 256, 0, s>>>(perm.p, rowid.p, val, nnz, at_colidx, at_val);
  LAGR_LAUNCH_CHECK();
  return LAGR_OK;
}

// Build (once) the row plan of a CSR: heavy rows and row blocks.  Every step runs on the device;
// the host reads four counts (two synchronisations).
int row_plan(RowPlan *pl, const int32_t *rowptr, int32_t n, cudaStream_t s, char *msg, int32_t units, int32_t hv,
             int32_t hchunk) {
  if (pl->nblk >= 0) return LAGR_OK;
  int32_t *heavy = nullptr, *blk = nullptr, *hc_off = nullptr, *hc_row = nullptr;
  uint8_t *hblk = nullptr;
  int32_t nheavy = 0, nblk = 0, nhc = 0;
  int st = LAGR_OK;
  {
    Temp<int32_t> hflag(s), hpos(s), ld(s), lp(s), b0(s), mark(s), mpos(s), nch(s);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    st = hflag.alloc(nn, msg, "heavy flags");
    if (st == LAGR_OK) st = hpos.alloc((size_t)n + 1, msg, "heavy positions");
    if (st == LAGR_OK) st = ld.alloc(nn, msg, "light degrees");
    if (st == LAGR_OK) st = lp.alloc((size_t)n + 1, msg, "light prefix");
    if (st == LAGR_OK) {
      row_classes<<<grid_for(n, 256), 256, 0, s>>>(rowptr, n, hv, hflag.p, ld.p);
      st = exclusive_scan(hflag.p, hpos.p, n, s, msg);
    }
    if (st == LAGR_OK) st = exclusive_scan(ld.p, lp.p, n, s, msg);
    int32_t light = 0;
    if (st == LAGR_OK) {
      const int32_t *src[2] = {hpos.p + n, lp.p + n};
      int32_t got[2];
      st = fetch_i32s(got, src, 2, s, msg);
      nheavy = got[0];
      light = got[1];
    }
    if (st == LAGR_OK) st = alloc_n(&heavy, (size_t)nheavy + 1, s, msg, "heavy row list");
    if (st == LAGR_OK && nheavy > 0) scatter_heavy<<<grid_for(n, 256), 256, 0, s>>>(hflag.p, hpos.p, n, heavy);
    // block starts: the first row at or after every units-th unit, plus each heavy row and the row
    // after it, so that every heavy row is a block of its own; marked per row, compacted by a scan
    const int64_t nb0 = ((int64_t)light + n) / units + 1;
    const int64_t ub64 = std::max<int64_t>(1, std::min<int64_t>(n, nb0 + 2 * (int64_t)nheavy));
    if (st == LAGR_OK) st = b0.alloc((size_t)nb0 + 1, msg, "row block starts");
    if (st == LAGR_OK) st = mark.alloc(nn, msg, "block marks");
    if (st == LAGR_OK) st = mpos.alloc((size_t)n + 1, msg, "block positions");
    if (st == LAGR_OK) st = alloc_n(&blk, (size_t)ub64 + 1, s, msg, "row blocks");
    if (st == LAGR_OK) st = alloc_n(&hblk, (size_t)ub64, s, msg, "heavy block flags");
    if (st == LAGR_OK) {
      block_starts<<<grid_for(nb0 + 1, 256), 256, 0, s>>>(lp.p, n, (int32_t)nb0, units, b0.p);
      const cudaError_t e = cudaMemsetAsync(mark.p, 0, nn * sizeof(int32_t), s);
      if (e != cudaSuccess) {
        set_msg(msg, "row plan: %s", cudaGetErrorString(e));
        st = LAGR_ERR_CUDA;
      }
    }
    if (st == LAGR_OK) {
      mark_cuts<<<grid_for(std::max<int64_t>(nb0, nheavy), 256), 256, 0, s>>>(b0.p, (int32_t)nb0, heavy, nheavy, n,
                                                                              mark.p);
      st = exclusive_scan(mark.p, mpos.p, n, s, msg);
    }
    if (st == LAGR_OK)
      scatter_blocks<<<grid_for(n, 256), 256, 0, s>>>(mark.p, mpos.p, rowptr, n, hv, blk, hblk);
    // chunks of the heavy rows
    if (st == LAGR_OK && nheavy > 0) {
      st = nch.alloc(nheavy, msg, "heavy chunk counts");
      if (st == LAGR_OK) st = alloc_n(&hc_off, (size_t)nheavy + 1, s, msg, "heavy chunk offsets");
      if (st == LAGR_OK) {
        heavy_chunk_counts<<<grid_for(nheavy, 256), 256, 0, s>>>(rowptr, heavy, nheavy, hchunk, nch.p);
        st = exclusive_scan(nch.p, hc_off, nheavy, s, msg);
      }
    }
    if (st == LAGR_OK) {
      const int32_t *src[2] = {mpos.p + n, nheavy > 0 ? hc_off + nheavy : mpos.p + n};
      int32_t got[2];
      st = fetch_i32s(got, src, 2, s, msg);
      nblk = n > 0 ? got[0] : 1;
      nhc = nheavy > 0 ? got[1] : 0;
    }
    if (st == LAGR_OK && nheavy > 0) {
      st = alloc_n(&hc_row, (size_t)(nhc > 0 ? nhc : 1), s, msg, "heavy chunk rows");
      if (st == LAGR_OK) heavy_chunk_rows<<<grid_for(nheavy, 256), 256, 0, s>>>(hc_off, nheavy, hc_row);
    }
    if (st == LAGR_OK) {
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        set_msg(msg, "row plan: %s", cudaGetErrorString(e));
        st = LAGR_ERR_CUDA;
      }
    }
  }
  if (st < 0) {
    dev_free(heavy, s);
    dev_free(blk, s);
    dev_free(hc_off, s);
    dev_free(hc_row, s);
    dev_free(hblk, s);
    return st;
  }
  pl->heavy = heavy;
  pl->nheavy = nheavy;
  pl->blk = blk;
  pl->nblk = nblk;
  pl->hc_off = hc_off;
  pl->hc_row = hc_row;
  pl->nhc = nhc;
  pl->hblk = hblk;
  pl->units = units;
  pl->heavy_len = hv;
  pl->hchunk = hchunk;
  return LAGR_OK;
}

}  // namespace lagr
