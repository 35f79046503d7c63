// bin.cu -- (a0) particle binning by bulk cell: the per-step particle to
// cell connectivity of Sec. 2.2 of arXiv 1807.11834.
//
// Cell rule (per axis): clamp(floor((x - x0) / H), 0, n_b - 1) with the
// quotient in IEEE double (subtract, then correctly rounded divide).  The
// FP32 path evaluates the quotient in float with a proven error bound and
// falls back to the exact double evaluation only when the float quotient
// lies within that bound of an integer, so the cell is bit-identical to the
// double rule at FP32 cost.
//
// The result is the stable order (ids ascending within each cell), built by
// one of two sorts that give identical bins:
//
// Per-cell sort (the default up to 2^23 particles and 32 per bulk cell on
// average; batched instances take it on request): the count atomics hand out
// arrival ranks, the scan of the counts gives the cell starts, each
// particle is placed at start + rank, and each cell's ids are then sorted
// (details below, before the kernels).
//
// Digit sort: least-significant-digit counting sort, one to three passes of
// at most 11 bits.  Each 4096-particle tile ranks its keys stably with
// warp-level match: warp w owns a contiguous 512-particle slice, walks it
// 32 at a time in index order and keeps per-digit counters in shared
// memory, so the rank of a particle within its digit group follows its
// index.  Tile histograms are scanned digit-major across tiles, which makes
// the whole pass stable and fully deterministic (no atomics decide any
// position).  Per-cell counts use integer atomics (order-independent), then
// a scan.
#include <algorithm>

#include "cg_internal.cuh"
#include "batch.cuh"

namespace cg {

__device__ __forceinline__ void add_status(unsigned long long* st, int outside, int nonfin) {
    // block-level aggregation by the caller; one atomic per non-zero counter
    if (outside) {
        atomicAdd(&st[ST_OUTSIDE], (unsigned long long)outside);
        atomicOr(&st[ST_FLAGS], (unsigned long long)CG_FLAG_OUTSIDE);
    }
    if (nonfin) {
        atomicAdd(&st[ST_NONFINITE], (unsigned long long)nonfin);
        atomicOr(&st[ST_FLAGS], (unsigned long long)CG_FLAG_NONFINITE);
    }
}

// ----------------------------------------------------------------------
// Key kernel: cell per particle, per-cell counts, tile histogram of digit 0
// ----------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void bin_key_body(const T* __restrict__ pos, long long n, const GridDev& g,
                                             int32_t* __restrict__ key, int32_t* __restrict__ count,
                                             int32_t* __restrict__ hist, int ntiles, int bits0, T* __restrict__ vol,
                                             unsigned long long* __restrict__ status, int* sh, Blk blk,
                                             double* __restrict__ eps_fill = nullptr, T* __restrict__ rec_fill = nullptr,
                                             T* __restrict__ eps_t_fill = nullptr) {
    __shared__ int s_cnt[2];
    const int R = 1 << bits0;
    for (int i = threadIdx.x; i < R; i += blockDim.x) sh[i] = 0;
    if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    int n_out = 0, n_nf = 0;
    const long long base = blk.id * kSortTile;
    V4<T> pv[kSortItems];
    // all position loads of the thread first, so they are in flight together
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        long long p = base + (long long)k * kSortThreads + threadIdx.x;
        if (p < n) pv[k] = ld4(pos, p);
    }
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        long long p = base + (long long)k * kSortThreads + threadIdx.x;
        bool valid = p < n;
        int c = -1;
        if (valid) {
            const V4<T>& v = pv[k];
            int outside = 0;
            if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) n_nf++;
            c = cell_of(v, g, outside);
            n_out += outside;
            key[p] = c;
            vol[p] = v.w;   // the diameter: the porosity forms the volume as an exact pair
        }
        // counts: one integer atomic per run of equal cells in the warp
        // (spatially ordered input has runs of several particles)
        const int len = run_head_length(c, valid);
        if (len) {
            atomicAdd(&count[c], len);
            atomicAdd(&sh[c & (R - 1)], len);
        }
    }
    if (n_out) atomicAdd(&s_cnt[0], n_out);
    if (n_nf) atomicAdd(&s_cnt[1], n_nf);
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += blockDim.x) hist[(long long)i * ntiles + blk.id] = sh[i];
    if (threadIdx.x == 0) add_status(status, s_cnt[0], s_cnt[1]);
    // the porosity of cells without particles is 1: set every cell here (and
    // the porosity of the drag record and of its path-precision copy), the
    // deposit overwrites the occupied ones (saves launches in the step)
    if (eps_fill)
        for (long long c = blk.id * blockDim.x + threadIdx.x; c < g.nbulk; c += blk.n * blockDim.x) {
            eps_fill[c] = 1.0;
            if (rec_fill) rec_fill[4 * c] = T(1);
            if (eps_t_fill) eps_t_fill[c] = T(1);
        }
}

template <typename T>
__global__ void __launch_bounds__(kSortThreads)
k_bin_key(const T* __restrict__ pos, long long n, GridDev g, int32_t* __restrict__ key,
          int32_t* __restrict__ count, int32_t* __restrict__ hist, int ntiles, int bits0,
          T* __restrict__ vol, unsigned long long* __restrict__ status, double* __restrict__ eps_fill,
          T* __restrict__ rec_fill, T* __restrict__ eps_t_fill) {
    pdl_wait();
    extern __shared__ int sh[];
    bin_key_body<T>(pos, n, g, key, count, hist, ntiles, bits0, vol, status, sh, launch_blk(), eps_fill, rec_fill,
                    eps_t_fill);
}

// Key kernel of the per-cell sort: cell, diameter and arrival rank of every
// particle, per-cell counts, porosity fill.  No shared memory and no block
// barrier; a block takes 4 x (its threads) particles, four per thread,
// consecutive lanes on consecutive particles (so runs of equal cells share
// one count atomic), and the thread's count atomics are issued together so
// their round trips overlap.

template <typename T>
__device__ __forceinline__ void bin_key_rank_body(const T* __restrict__ pos, long long n, const GridDev& g,
                                                  int32_t* __restrict__ key, int32_t* __restrict__ count,
                                                  T* __restrict__ vol, unsigned long long* __restrict__ status,
                                                  double* __restrict__ eps_fill, T* __restrict__ rec_fill,
                                                  T* __restrict__ eps_t_fill, int32_t* __restrict__ arrival, Blk blk) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long base = blk.id * (long long)(blockDim.x * kKeyItems);
    V4<T> pv[kKeyItems];
#pragma unroll
    for (int k = 0; k < kKeyItems; ++k) {
        const long long p = base + k * blockDim.x + threadIdx.x;
        if (p < n) pv[k] = ld4(pos, p);
    }
    int n_out = 0, n_nf = 0;
    int ck[kKeyItems], lk[kKeyItems], old[kKeyItems];
#pragma unroll
    for (int k = 0; k < kKeyItems; ++k) {
        const long long p = base + k * blockDim.x + threadIdx.x;
        const bool valid = p < n;
        int c = -1;
        if (valid) {
            const V4<T>& v = pv[k];
            int outside = 0;
            if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) n_nf++;
            c = cell_of(v, g, outside);
            n_out += outside;
            key[p] = c;
            vol[p] = v.w;   // the diameter: the porosity forms the volume as an exact pair
        }
        ck[k] = c;
        lk[k] = run_head_length(c, valid);
    }
#pragma unroll
    for (int k = 0; k < kKeyItems; ++k) old[k] = lk[k] ? atomicAdd(&count[ck[k]], lk[k]) : 0;
    // the run's head took len slots of the cell's arrival order; every
    // member finds its head (the last head at or below it)
#pragma unroll
    for (int k = 0; k < kKeyItems; ++k) {
        const long long p = base + k * blockDim.x + threadIdx.x;
        const unsigned heads = __ballot_sync(full, lk[k] != 0);
        const int head = 31 - __clz(heads & ((2u << lane) - 1u));
        const int o = __shfl_sync(full, old[k], head < 0 ? 0 : head);
        if (p < n) arrival[p] = o + lane - head;
    }
    n_out = __reduce_add_sync(full, n_out);
    n_nf = __reduce_add_sync(full, n_nf);
    if (lane == 0 && (n_out | n_nf)) add_status(status, n_out, n_nf);
    // the porosity of cells without particles is 1: set every cell here (and
    // the porosity of the drag record and of its path-precision copy), the
    // deposit overwrites the occupied ones
    if (eps_fill)
        for (long long c = blk.id * blockDim.x + threadIdx.x; c < g.nbulk; c += blk.n * blockDim.x) {
            eps_fill[c] = 1.0;
            if (rec_fill) rec_fill[4 * c] = T(1);
            if (eps_t_fill) eps_t_fill[c] = T(1);
        }
}

template <typename T>
__global__ void __launch_bounds__(kKeyThreads, 5)
k_bin_key_rank(const T* __restrict__ pos, long long n, GridDev g, int32_t* __restrict__ key,
               int32_t* __restrict__ count, T* __restrict__ vol, unsigned long long* __restrict__ status,
               double* __restrict__ eps_fill, T* __restrict__ rec_fill, T* __restrict__ eps_t_fill,
               int32_t* __restrict__ arrival) {
    pdl_wait();
    bin_key_rank_body<T>(pos, n, g, key, count, vol, status, eps_fill, rec_fill, eps_t_fill, arrival, launch_blk());
}

// Tile histogram of a digit of already-computed keys (second pass).
__device__ __forceinline__ void bin_hist_body(const int32_t* __restrict__ keys, long long n, int ntiles, int shift,
                                              int bits, int32_t* __restrict__ hist, int* sh, Blk blk) {
    const int R = 1 << bits;
    for (int i = threadIdx.x; i < R; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const long long base = blk.id * kSortTile;
#pragma unroll 4
    for (int k = 0; k < kSortItems; ++k) {
        long long p = base + (long long)k * kSortThreads + threadIdx.x;
        bool valid = p < n;
        if (valid) atomicAdd(&sh[(__ldg(keys + p) >> shift) & (R - 1)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += blockDim.x) hist[(long long)i * ntiles + blk.id] = sh[i];
}

__global__ void __launch_bounds__(kSortThreads)
k_bin_hist(const int32_t* __restrict__ keys, long long n, int ntiles, int shift, int bits,
           int32_t* __restrict__ hist) {
    pdl_wait();
    extern __shared__ int sh[];
    bin_hist_body(keys, n, ntiles, shift, bits, hist, sh, launch_blk());
}

// Stable scatter of one digit pass.  offs = exclusive scan of the tile
// histograms, digit-major ([digit][tile]).  The tile is first ranked (each
// warp walks its 512-element slice in order with match_any and per-warp
// digit counters), then reordered by digit in shared memory, and finally
// written out slot by slot: consecutive threads write consecutive addresses
// of each digit's run, so the stores coalesce even for keys in random order.
// Shared memory (ints): a region holding first the per-warp counters
// [kSortWarps][R], then the staged tile (keys, ids, diameters); then the
// tile-local digit starts [R] and the global shifts [R].

template <bool FIRST, bool FINAL, typename T>
__device__ __forceinline__ void bin_scatter_body(const int32_t* __restrict__ keys_in,
                                                 const int32_t* __restrict__ vals_in, long long n, int ntiles,
                                                 int shift, int bits, const int32_t* __restrict__ offs,
                                                 int32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out,
                                                 int32_t* __restrict__ perm, int32_t* __restrict__ key_sorted,
                                                 int32_t* __restrict__ inv_perm, const T* __restrict__ vol,
                                                 T* __restrict__ vol_sorted, int* smem, Blk blk) {
    __shared__ int shw[32];
    const int R = 1 << bits;
    const size_t region = ((size_t)kSortWarps << bits) > (size_t)kSortTile * (8 + sizeof(T)) / sizeof(int)
                              ? ((size_t)kSortWarps << bits)
                              : (size_t)kSortTile * (8 + sizeof(T)) / sizeof(int);
    int* cnt = smem;                       // [kSortWarps][R], then the staged tile
    int* lbase = smem + region;            // [R] tile-local start of each digit
    int* shiftg = lbase + R;               // [R] global start - local start
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kSortWarps * R; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    int* wc = cnt + warp * R;
    const unsigned lt = lanemask_lt();
    const long long tile0 = blk.id * kSortTile;
    const long long base = tile0 + (long long)warp * (kSortTile / kSortWarps);
    const int tile_n = (int)(n - tile0 < kSortTile ? n - tile0 : kSortTile);
    int kv[kSortItems], vv[kSortItems], rk[kSortItems];
    T vol_k[kSortItems];
    // all loads of the slice first, so they are in flight together
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        long long p = base + k * 32 + lane;
        bool valid = p < n;
        kv[k] = valid ? __ldg(keys_in + p) : 0;
        vv[k] = valid ? (FIRST ? (int)p : __ldg(vals_in + p)) : 0;
    }
    if (FINAL)
#pragma unroll
        for (int k = 0; k < kSortItems; ++k)
            if (base + k * 32 + lane < n) vol_k[k] = __ldg(vol + vv[k]);
    // rank within the warp's slice, in index order
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        long long p = base + k * 32 + lane;
        bool valid = p < n;
        int kk = kv[k];
        int d = valid ? ((kk >> shift) & (R - 1)) : -1;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = __popc(peers & lt);
        int c0 = valid ? wc[d] : 0;
        __syncwarp();
        if (valid && before == 0) wc[d] = c0 + __popc(peers);
        __syncwarp();
        rk[k] = c0 + before;
    }
    __syncthreads();
    // per digit: the warps' exclusive offsets within the tile's digit run,
    // and the digit's count; then the tile-local digit starts (a block scan
    // over the digits, consecutive digits per thread)
    constexpr int kMaxPer = (1 << kMaxDigitBits) / kSortThreads;   // digits per thread at most
    const int per = (R + (int)blockDim.x - 1) / (int)blockDim.x;
    int tot[kMaxPer > 0 ? kMaxPer : 1];
    int mysum = 0;
#pragma unroll
    for (int j = 0; j < (kMaxPer > 0 ? kMaxPer : 1); ++j) {
        tot[j] = 0;
        const int d = threadIdx.x * per + j;
        if (j < per && d < R) {
            int run = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                const int t = cnt[w * R + d];
                cnt[w * R + d] = run;
                run += t;
            }
            tot[j] = run;
            mysum += run;
        }
    }
    int all;
    int ex = block_exclusive_scan(mysum, shw, all);
#pragma unroll
    for (int j = 0; j < (kMaxPer > 0 ? kMaxPer : 1); ++j) {
        const int d = threadIdx.x * per + j;
        if (j < per && d < R) {
            lbase[d] = ex;
            shiftg[d] = __ldg(offs + (long long)d * ntiles + blk.id) - ex;
            ex += tot[j];
        }
    }
    __syncthreads();
    // local slot of every element
    int lp[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        long long p = base + k * 32 + lane;
        lp[k] = -1;
        if (p < n) {
            const int d = (kv[k] >> shift) & (R - 1);
            lp[k] = lbase[d] + wc[d] + rk[k];
        }
    }
    __syncthreads();   // every counter read: the region now takes the staged tile
    int* sk = cnt;
    int* sv = cnt + kSortTile;
    T* svol = reinterpret_cast<T*>(cnt + 2 * kSortTile);
#pragma unroll
    for (int k = 0; k < kSortItems; ++k)
        if (lp[k] >= 0) {
            sk[lp[k]] = kv[k];
            sv[lp[k]] = vv[k];
            if (FINAL) svol[lp[k]] = vol_k[k];
        }
    __syncthreads();
    // write out in slot order: each digit's run is contiguous in memory
    for (int i = threadIdx.x; i < tile_n; i += blockDim.x) {
        const int key = sk[i];
        const int val = sv[i];
        const int dst = i + shiftg[(key >> shift) & (R - 1)];
        if (FINAL) {
            perm[dst] = val;
            key_sorted[dst] = key;
            inv_perm[val] = dst;
            vol_sorted[dst] = svol[i];
        } else {
            keys_out[dst] = key;
            vals_out[dst] = val;
        }
    }
}

template <bool FIRST, bool FINAL, typename T>
__global__ void __launch_bounds__(kSortThreads, 2)
k_bin_scatter(const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in, long long n,
              int ntiles, int shift, int bits, const int32_t* __restrict__ offs,
              int32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out, int32_t* __restrict__ perm,
              int32_t* __restrict__ key_sorted, int32_t* __restrict__ inv_perm, const T* __restrict__ vol,
              T* __restrict__ vol_sorted) {
    pdl_wait();
    extern __shared__ int cnt[];
    bin_scatter_body<FIRST, FINAL, T>(keys_in, vals_in, n, ntiles, shift, bits, offs, keys_out, vals_out, perm,
                                      key_sorted, inv_perm, vol, vol_sorted, cnt, launch_blk());
}

// ----------------------------------------------------------------------
// Exclusive scan of int32 (totals fit in int32: at most 2^31 - 1 particles)
// ----------------------------------------------------------------------

// Load the 16 consecutive elements of a thread (zero past m).
__device__ __forceinline__ void load16(const int32_t* __restrict__ in, long long start, long long m, int v[16]) {
    if (start + 16 <= m) {
        const int4* q = reinterpret_cast<const int4*>(in + start);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int4 t = q[j];
            v[4 * j] = t.x; v[4 * j + 1] = t.y; v[4 * j + 2] = t.z; v[4 * j + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = (start + j < m) ? in[start + j] : 0;
    }
}

// Block `id` of a job is block `blk` of array `which`; `first` is the job's
// index of that array's first block.
__device__ __forceinline__ void scan_locate(const ScanJob& j, long long id, int& which, long long& blk,
                                            long long& first) {
    blk = id;
    which = 0;
    first = 0;
    while (which < kScanArrays - 1 && blk >= j.nblk[which]) {
        blk -= j.nblk[which];
        first += j.nblk[which];
        ++which;
    }
}

// Blocks of a job: [0, nblk[0]) over array 0, then nblk[1] over array 1,
// then nblk[2] over array 2; part holds one total per block of the job.
__device__ __forceinline__ void scan_reduce_body(const ScanJob& j, int32_t* __restrict__ part, Blk b) {
    __shared__ int shw[32];
    int which;
    long long blk, first;
    scan_locate(j, b.id, which, blk, first);
    long long start = blk * kScanItems + threadIdx.x * 16;
    int v[16];
    load16(j.in[which], start, j.m[which], v);
    int s = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += v[k];
    int total;
    block_exclusive_scan(s, shw, total);
    if (threadIdx.x == 0) part[b.id] = total;
}

__global__ void __launch_bounds__(256) k_scan_reduce(ScanJob j, int32_t* __restrict__ part) {
    pdl_wait();
    if (j.skip && __ldg(j.skip) == 0) return;
    scan_reduce_body(j, part, launch_blk());
}

// Each block sums the partials of the blocks before it in its array (a few
// thousand at most), then scans its own chunk: no third launch.
__device__ __forceinline__ void scan_down_body(const ScanJob& j, const int32_t* __restrict__ part, Blk b) {
    __shared__ int shw[32];
    __shared__ int s_base;
    int which;
    long long blk, first;
    scan_locate(j, b.id, which, blk, first);
    int acc = 0;
    for (long long i = threadIdx.x; i < blk; i += blockDim.x) acc += part[first + i];
    int tot;
    block_exclusive_scan(acc, shw, tot);
    if (threadIdx.x == 0) s_base = tot;
    __syncthreads();
    const int base = s_base;
    long long start = blk * kScanItems + threadIdx.x * 16;
    int v[16];
    load16(j.in[which], start, j.m[which], v);
    int s = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += v[k];
    int total;
    int ex = block_exclusive_scan(s, shw, total) + base;
    int32_t* out = j.out[which];
    const long long m = j.m[which];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (start + k < m) out[start + k] = ex;
        ex += v[k];
    }
}

__global__ void __launch_bounds__(256) k_scan_down(ScanJob j, const int32_t* __restrict__ part) {
    pdl_wait();
    if (j.skip && __ldg(j.skip) == 0) return;
    scan_down_body(j, part, launch_blk());
}

// Exclusive scans of up to three arrays by one pair of launches (out may
// alias in; an array with in == nullptr is skipped).  skip (device, may be
// null): when it reads 0 the launches return at once, the caller having
// left the outputs in their scanned form.
cg_status scan_exclusive(cg_grids* g, int count, const int32_t* const* in, int32_t* const* out, const long long* m,
                         const int32_t* skip) {
    ScanJob j;
    j.skip = skip;
    long long nblk = 0;
    for (int a = 0; a < kScanArrays; ++a) {
        const bool use = a < count && in[a];
        j.in[a] = use ? in[a] : nullptr;
        j.out[a] = use ? out[a] : nullptr;
        j.m[a] = use ? m[a] : 0;
        j.nblk[a] = (j.m[a] + kScanItems - 1) / kScanItems;
        nblk += j.nblk[a];
    }
    if (nblk == 0) return CG_OK;
    if (nblk > g->scan_cap) return CG_ERR_OUT_OF_RANGE;
    CG_LAUNCH(g, "bin_scan", k_scan_reduce, (unsigned)nblk, 256, 0, j, g->scan_part);
    CG_LAUNCH(g, "bin_scan", k_scan_down, (unsigned)nblk, 256, 0, j, g->scan_part);
    return CG_OK;
}

static cg_status scan_exclusive2(cg_grids* g, const int32_t* inA, int32_t* outA, long long mA,
                                 const int32_t* inB, int32_t* outB, long long mB) {
    const int32_t* in[2] = {inA, inB};
    int32_t* out[2] = {outA, outB};
    const long long m[2] = {mA, mB};
    return scan_exclusive(g, 2, in, out, m);
}


// ----------------------------------------------------------------------
// Default sort: arrival rank, placement, and a sort of every cell's ids.
//
// The key kernel's count atomics hand each particle its arrival rank within
// its cell; after the scan of the counts, slot = start(cell) + rank places
// every particle in its cell's segment, in an order the atomics decided.
// Sorting each segment by particle id then gives exactly the stable order
// (ids ascending within a cell), independent of that arrival order.  Cells
// of up to 256 particles are sorted by one warp in registers (bitonic
// network); larger ones by a whole CTA, in least-significant-digit passes
// over the ids.  Placement and the per-cell sort touch memory at random
// where the caller's particle order is random, so this sort suits orders
// that keep neighbours close (as DEM codes keep theirs); the digit sort
// above moves whole digit runs and suits random orders.
// ----------------------------------------------------------------------

// Four particles per thread, consecutive lanes on consecutive particles
// (so runs of one cell's arrivals store to consecutive slots), with the
// thread's four loads, gathers and stores each in flight together.
__device__ __forceinline__ void place_body(const int32_t* __restrict__ key, const int32_t* __restrict__ arrival,
                                           const int32_t* __restrict__ cell_start, long long n,
                                           int32_t* __restrict__ tmp, Blk blk) {
    constexpr int U = kPlaceItems;
    const long long span = (long long)blockDim.x * U;
    for (long long b0 = blk.id * span; b0 < n; b0 += blk.n * span) {
        int kk[U], aa[U], st[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const long long p = b0 + j * blockDim.x + threadIdx.x;
            kk[j] = p < n ? __ldg(key + p) : 0;
            aa[j] = p < n ? __ldg(arrival + p) : 0;
        }
#pragma unroll
        for (int j = 0; j < U; ++j) st[j] = __ldg(cell_start + kk[j]);
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const long long p = b0 + j * blockDim.x + threadIdx.x;
            if (p < n) tmp[st[j] + aa[j]] = (int)p;
        }
    }
}

// run_if (nullable): the kernel does nothing unless *run_if is non-zero
// (the fallback of the incremental rebinning, decided on the device).
__global__ void __launch_bounds__(512) k_bin_place(const int32_t* __restrict__ key,
                                                   const int32_t* __restrict__ arrival,
                                                   const int32_t* __restrict__ cell_start, long long n,
                                                   int32_t* __restrict__ tmp, const int32_t* __restrict__ run_if) {
    pdl_wait();
    if (run_if && *run_if == 0) return;
    place_body(key, arrival, cell_start, n, tmp, launch_blk());
}

// Ascending bitonic sort of the warp's 32*K values, blocked layout: lane l
// holds elements l*K .. l*K + K - 1.  Partners closer than K are in the
// same thread; farther ones are exchanged by shuffles.
template <int K>
__device__ __forceinline__ void warp_bitonic(int (&v)[K]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32 * K; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < K) {
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    const int q = r ^ j;
                    if (q > r) {
                        const bool asc = ((lane * K + r) & k) == 0;
                        const int a = v[r], b = v[q];
                        v[r] = asc ? min(a, b) : max(a, b);
                        v[q] = asc ? max(a, b) : min(a, b);
                    }
                }
            } else {
                const int lj = j / K;
                const bool lower = (lane & lj) == 0;
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    const bool asc = ((lane * K + r) & k) == 0;
                    const int o = __shfl_xor_sync(0xffffffffu, v[r], lj);
                    v[r] = (lower == asc) ? min(v[r], o) : max(v[r], o);
                }
            }
        }
    }
}

// Outputs of one sorted slot: the id, its cell, its inverse, its diameter.
template <typename T>
__device__ __forceinline__ void emit_slot(long long slot, int id, int cell, int32_t* __restrict__ perm,
                                          int32_t* __restrict__ key_sorted, int32_t* __restrict__ inv_perm,
                                          const T* __restrict__ vol, T* __restrict__ vol_sorted) {
    perm[slot] = id;
    key_sorted[slot] = cell;
    inv_perm[id] = (int)slot;
    vol_sorted[slot] = __ldg(vol + id);
}

// Sort the c (<= 32 K) ids at src (shared memory when staged, else global)
// with one warp; staged: write them back sorted and write their cells,
// else write all outputs of the slots s_out .. s_out + c - 1.
template <int K, typename T>
__device__ __forceinline__ void warp_sort_cell(int32_t* src, bool staged, long long s_out, int c, int cell,
                                               int32_t* __restrict__ perm, int32_t* __restrict__ key_sorted,
                                               int32_t* __restrict__ inv_perm, const T* __restrict__ vol,
                                               T* __restrict__ vol_sorted) {
    const int lane = threadIdx.x & 31;
    int v[K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int e = lane * K + r;
        v[r] = e < c ? src[e] : 0x7fffffff;
    }
    if (c > 1) warp_bitonic<K>(v);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int e = lane * K + r;
        if (e < c) {
            if (staged) {
                src[e] = v[r];
                key_sorted[s_out + e] = cell;
            } else {
                emit_slot<T>(s_out + e, v[r], cell, perm, key_sorted, inv_perm, vol, vol_sorted);
            }
        }
    }
}

// One warp sorts the ids of a cell larger than kSegWarpMax: passes of 8-bit
// digits of (id - min id), each a histogram, a scan of the 256 digit counts,
// and a stable scatter that walks the ids 32 at a time in index order (rank
// within a digit by match_any, running digit starts in shared memory).  Ids
// move between buf0 and buf1 (the same slots of two arrays); the outputs
// are written from whichever holds the last pass.  sm: 256 ints of the
// warp's shared memory.
template <typename T>
__device__ __noinline__ void warp_big_sort(int cell, long long s, int c, int32_t* buf0, int32_t* buf1, int* sm,
                                           int32_t* __restrict__ perm, int32_t* __restrict__ key_sorted,
                                           int32_t* __restrict__ inv_perm, const T* __restrict__ vol,
                                           T* __restrict__ vol_sorted) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int lo = 0x7fffffff, hi = 0;
    for (int i = lane; i < c; i += 32) {
        const int v = buf0[s + i];
        lo = min(lo, v);
        hi = max(hi, v);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(full, lo, off));
        hi = max(hi, __shfl_xor_sync(full, hi, off));
    }
    const unsigned span = (unsigned)(hi - lo);
    int passes = 0;
    while (passes < 4 && (span >> (8 * passes)) != 0u) ++passes;
    int32_t* in = buf0;
    int32_t* out = buf1;
    const unsigned lt = lanemask_lt();
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = 8 * ps;
#pragma unroll
        for (int j = 0; j < 8; ++j) sm[lane * 8 + j] = 0;
        __syncwarp();
        for (int i = lane; i < c; i += 32) atomicAdd(&sm[((unsigned)(in[s + i] - lo) >> shift) & 255u], 1);
        __syncwarp();
        // exclusive scan of the 256 counts: 8 consecutive digits per lane
        int cnt[8], tot = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            cnt[j] = sm[lane * 8 + j];
            tot += cnt[j];
        }
        int x = tot;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(full, x, off);
            if (lane >= off) x += y;
        }
        int run = x - tot;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            sm[lane * 8 + j] = run;
            run += cnt[j];
        }
        __syncwarp();
        for (int base = 0; base < c; base += 32) {
            const int e = base + lane;
            const bool valid = e < c;
            const int v = valid ? in[s + e] : 0;
            const int d = valid ? (int)(((unsigned)(v - lo) >> shift) & 255u) : -1;
            const unsigned peers = __match_any_sync(full, d);
            const int before = __popc(peers & lt);
            const int start = valid ? sm[d] : 0;
            __syncwarp();
            if (valid && before == 0) sm[d] = start + __popc(peers);
            __syncwarp();
            if (valid) out[s + start + before] = v;
        }
        __syncwarp();
        int32_t* t = in;
        in = out;
        out = t;
    }
    for (int i = lane; i < c; i += 32) emit_slot<T>(s + i, in[s + i], cell, perm, key_sorted, inv_perm, vol, vol_sorted);
    __syncwarp();
}


// Each warp goes through groups of kGroupCells consecutive cells on its
// own (no CTA-wide barrier): warp w of nw takes groups w, w + nw, w + 2nw,
// ..., so occupied groups spread over every warp even where the particles
// fill a small part of the grid; lane l first checks group w + l nw (of the
// next 32) for particles, so empty groups cost one lookup per 32.  A group
// of at most kWarpStage ids is read into the warp's shared memory with
// coalesced loads; the warp sorts its cells there one after another (in
// registers) and writes them back, then writes the group's outputs slot by
// slot (coalesced, with the diameter gathers of the lane's slots in flight
// together).  A larger group's cells are sorted straight from global
// memory.  Cells of more than kSegWarpMax particles are sorted by
// warp_big_sort after the group's other cells are written.
template <typename T>
__device__ __forceinline__ void seg_sort_body(const int32_t* __restrict__ cell_start, long long nbulk, int32_t* tmp,
                                              int32_t* alt, int32_t* __restrict__ perm,
                                              int32_t* __restrict__ key_sorted, int32_t* __restrict__ inv_perm,
                                              const T* __restrict__ vol, T* __restrict__ vol_sorted, Blk blk) {
    __shared__ int s_stage[kSegSortWarps][kWarpStage];
    const unsigned full = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* stage = s_stage[warp];
    const long long nw = blk.n * kSegSortWarps;
    const long long w = blk.id * kSegSortWarps + warp;
    const long long ngroups = (nbulk + kGroupCells - 1) / kGroupCells;
    for (long long gsup = w; gsup < ngroups; gsup += 32 * nw) {
        bool ne = false;
        {
            const long long gi = gsup + lane * nw;
            if (gi < ngroups) {
                const long long c0 = gi * kGroupCells;
                const long long c1 = c0 + kGroupCells < nbulk ? c0 + kGroupCells : nbulk;
                ne = __ldg(cell_start + c1) != __ldg(cell_start + c0);
            }
        }
        unsigned todo = __ballot_sync(full, ne);
        while (todo) {
            const int k = __ffs(todo) - 1;
            todo &= todo - 1;
            const long long c0 = (gsup + k * nw) * kGroupCells;
            const int nc = (int)(c0 + kGroupCells < nbulk ? kGroupCells : nbulk - c0);
            const int csl = lane <= nc ? __ldg(cell_start + c0 + lane) : 0;   // lane j: start of cell j
            const int s0 = __shfl_sync(full, csl, 0);
            const int m = __shfl_sync(full, csl, nc) - s0;
            const bool staged = m <= kWarpStage;
            if (staged) {
                for (int i = lane; i < m; i += 32) stage[i] = tmp[(long long)s0 + i];
                __syncwarp();
            }
            unsigned bigs = 0;
            for (int j = 0; j < nc; ++j) {
                const int a = __shfl_sync(full, csl, j) - s0;
                const int c = __shfl_sync(full, csl, j + 1) - s0 - a;
                const int cell = (int)(c0 + j);
                int32_t* src = staged ? stage + a : tmp + s0 + a;
                if (c == 0) continue;
                if (c > kSegWarpMax) {
                    bigs |= 1u << j;
                    if (staged)   // its slots are written by warp_big_sort
                        for (int e = lane; e < c; e += 32) src[e] = -1;
                } else if (c <= 32) {
                    warp_sort_cell<1, T>(src, staged, s0 + a, c, cell, perm, key_sorted, inv_perm, vol, vol_sorted);
                } else if (c <= 64) {
                    warp_sort_cell<2, T>(src, staged, s0 + a, c, cell, perm, key_sorted, inv_perm, vol, vol_sorted);
                } else if (c <= 128) {
                    warp_sort_cell<4, T>(src, staged, s0 + a, c, cell, perm, key_sorted, inv_perm, vol, vol_sorted);
                } else {
                    warp_sort_cell<8, T>(src, staged, s0 + a, c, cell, perm, key_sorted, inv_perm, vol, vol_sorted);
                }
            }
            __syncwarp();
            if (staged) {
                constexpr int U = 4;
                for (int i0 = lane; i0 < m; i0 += U * 32) {
                    int id[U];
                    T d[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int i = i0 + u * 32;
                        id[u] = i < m ? stage[i] : -1;
                        if (id[u] >= 0) d[u] = __ldg(vol + id[u]);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const long long slot = (long long)s0 + i0 + u * 32;
                        if (id[u] >= 0) {
                            perm[slot] = id[u];
                            inv_perm[id[u]] = (int)slot;
                            vol_sorted[slot] = d[u];
                        }
                    }
                }
                __syncwarp();
            }
            while (bigs) {
                const int j = __ffs(bigs) - 1;
                bigs &= bigs - 1;
                const int a = __shfl_sync(full, csl, j);
                const int c = __shfl_sync(full, csl, j + 1) - a;
                warp_big_sort<T>((int)(c0 + j), a, c, tmp, alt, stage, perm, key_sorted, inv_perm, vol, vol_sorted);
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kSegSortWarps * 32, 4)
k_seg_sort(const int32_t* __restrict__ cell_start, long long nbulk, int32_t* tmp, int32_t* alt,
           int32_t* __restrict__ perm, int32_t* __restrict__ key_sorted, int32_t* __restrict__ inv_perm,
           const T* __restrict__ vol, T* __restrict__ vol_sorted, const int32_t* __restrict__ run_if) {
    pdl_wait();
    if (run_if && *run_if == 0) return;
    seg_sort_body<T>(cell_start, nbulk, tmp, alt, perm, key_sorted, inv_perm, vol, vol_sorted, launch_blk());
}

static PerDeviceOnce g_attr_once;

static cg_status set_attrs() {
    return once_per_device(g_attr_once, [] {
        const int smem = (int)scatter_smem_bytes(kMaxDigitBits, sizeof(double));   // 144 KB at 2^11 digits
#define CG_ATTR(F, L, T) \
    CG_CUDA(cudaFuncSetAttribute(k_bin_scatter<F, L, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))
        CG_ATTR(true, true, float);
        CG_ATTR(true, false, float);
        CG_ATTR(false, true, float);
        CG_ATTR(false, false, float);
        CG_ATTR(true, true, double);
        CG_ATTR(true, false, double);
        CG_ATTR(false, true, double);
        CG_ATTR(false, false, double);
#undef CG_ATTR
        return CG_OK;
    });
}

template <typename T>
static cg_status bin_passes(cg_grids* g, long long n, const T* pos, int ntiles, long long m0, double* eps_fill,
                            T* rec_fill, T* eps_t_fill) {
    const long long nbulk = g->gd.nbulk;
    const int np = g->npasses;
    const int b0 = g->pass_bits[0];
    CG_LAUNCH(g, "bin_key", k_bin_key<T>, ntiles, kSortThreads, sizeof(int) << b0, pos, n, g->gd, g->key,
              g->cell_start, g->hist, ntiles, b0, (T*)g->vol, g->status, eps_fill, rec_fill, eps_t_fill);
    CG_TRY(scan_exclusive2(g, g->cell_start, g->cell_start, nbulk + 1, g->hist, g->hist, m0));
    // pass p reads (keys, ids) from in[p] and writes them to in[p + 1]; the
    // last pass writes the final order
    int32_t* ks[kMaxPasses + 1] = {g->key, g->key1, g->key2, nullptr};
    int32_t* vs[kMaxPasses + 1] = {nullptr, g->val1, g->val2, nullptr};
    int shift = 0;
    for (int p = 0; p < np; ++p) {
        const int bits = g->pass_bits[p];
        if (p > 0) {
            const long long m = (long long)ntiles << bits;
            CG_LAUNCH(g, "bin_hist", k_bin_hist, ntiles, kSortThreads, sizeof(int) << bits, ks[p], n, ntiles, shift,
                      bits, g->hist);
            CG_TRY(scan_exclusive2(g, g->hist, g->hist, m, nullptr, nullptr, 0));
        }
        const size_t smem = scatter_smem_bytes(bits, sizeof(T));
        const bool first = p == 0, last = p == np - 1;
        if (first && last)
            CG_LAUNCH(g, "bin_scatter", (k_bin_scatter<true, true, T>), ntiles, kSortThreads, smem, ks[0], nullptr,
                      n, ntiles, shift, bits, g->hist, nullptr, nullptr, g->perm, g->key_sorted, g->inv_perm,
                      (const T*)g->vol, (T*)g->vol_sorted);
        else if (first)
            CG_LAUNCH(g, "bin_scatter", (k_bin_scatter<true, false, T>), ntiles, kSortThreads, smem, ks[0], nullptr,
                      n, ntiles, shift, bits, g->hist, ks[1], vs[1], nullptr, nullptr, nullptr, (const T*)nullptr,
                      (T*)nullptr);
        else if (last)
            CG_LAUNCH(g, "bin_scatter", (k_bin_scatter<false, true, T>), ntiles, kSortThreads, smem, ks[p], vs[p],
                      n, ntiles, shift, bits, g->hist, nullptr, nullptr, g->perm, g->key_sorted, g->inv_perm,
                      (const T*)g->vol, (T*)g->vol_sorted);
        else
            CG_LAUNCH(g, "bin_scatter", (k_bin_scatter<false, false, T>), ntiles, kSortThreads, smem, ks[p], vs[p],
                      n, ntiles, shift, bits, g->hist, ks[p + 1], vs[p + 1], nullptr, nullptr, nullptr,
                      (const T*)nullptr, (T*)nullptr);
        shift += bits;
    }
    return CG_OK;
}

// Default sort: key + arrival rank, scan of the counts (two launches),
// placement, per-cell sort.
template <typename T>
static cg_status bin_rank(cg_grids* g, long long n, const T* pos, int ntiles, double* eps_fill, T* rec_fill,
                          T* eps_t_fill) {
    const long long nbulk = g->gd.nbulk;
    const long long kb = (n + kKeyThreads * kKeyItems - 1) / (kKeyThreads * kKeyItems);
    CG_LAUNCH(g, "bin_key", k_bin_key_rank<T>, (unsigned)kb, kKeyThreads, 0, pos, n, g->gd, g->key, g->cell_start,
              (T*)g->vol, g->status, eps_fill, rec_fill, eps_t_fill, g->key2);
    CG_TRY(scan_exclusive2(g, g->cell_start, g->cell_start, nbulk + 1, nullptr, nullptr, 0));
    return launch_cellsort_tail(g, n, g->cell_start, nullptr);
}

// Placement and per-cell sort of the per-cell sort, from the cell starts cs
// and the arrival ranks in key2 (the keys in key, the diameters in vol).
cg_status launch_cellsort_tail(cg_grids* g, long long n, const int32_t* cs, const int32_t* run_if) {
    const long long nbulk = g->gd.nbulk;
    // as the device's fallback (run_if set) the kernels are usually idle: one
    // grid-stride CTA per SM keeps an idle launch short
    const long long per_sm = run_if ? 1 : 4;
    const long long pb = std::min<long long>((n + 512 * kPlaceItems - 1) / (512 * kPlaceItems),
                                             (long long)g->num_sms * per_sm);
    CG_LAUNCH(g, "bin_place", k_bin_place, (unsigned)pb, 512, 0, g->key, g->key2, cs, n, g->val1, run_if);
    const long long sb = std::min<long long>((nbulk + kGroupCells * kSegSortWarps - 1) / (kGroupCells * kSegSortWarps),
                                             (long long)g->num_sms * per_sm);
    if (g->fp64)
        CG_LAUNCH(g, "bin_seg_sort", k_seg_sort<double>, (unsigned)sb, kSegSortWarps * 32, 0, cs, nbulk, g->val1,
                  g->key1, g->perm, g->key_sorted, g->inv_perm, (const double*)g->vol, (double*)g->vol_sorted, run_if);
    else
        CG_LAUNCH(g, "bin_seg_sort", k_seg_sort<float>, (unsigned)sb, kSegSortWarps * 32, 0, cs, nbulk, g->val1,
                  g->key1, g->perm, g->key_sorted, g->inv_perm, (const float*)g->vol, (float*)g->vol_sorted, run_if);
    return CG_OK;
}

// ----------------------------------------------------------------------
// Physical reorder into the binned order: slot s takes the records of
// particle perm[s] (16 or 32 bytes each; consecutive threads write
// consecutive slots).
// ----------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_reorder(const int32_t* __restrict__ perm, long long n,
                                                 const T* __restrict__ pos, const T* __restrict__ vel,
                                                 T* __restrict__ pos_out, T* __restrict__ vel_out) {
    pdl_wait();
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int p = __ldg(perm + s);
        const V4<T> a = ld4(pos, p);
        st4(pos_out, s, a.x, a.y, a.z, a.w);
        if (vel) {
            const V4<T> b = ld4(vel, p);
            st4(vel_out, s, b.x, b.y, b.z, b.w);
        }
    }
}

cg_status launch_reorder(cg_grids* g, long long n, const void* pos_d, const void* vel, void* pos_out, void* vel_out) {
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, (long long)g->num_sms * 16);
    if (g->fp64)
        CG_LAUNCH(g, "reorder", k_reorder<double>, grid, 256, 0, g->perm, n, (const double*)pos_d,
                  (const double*)vel, (double*)pos_out, (double*)vel_out);
    else
        CG_LAUNCH(g, "reorder", k_reorder<float>, grid, 256, 0, g->perm, n, (const float*)pos_d, (const float*)vel,
                  (float*)pos_out, (float*)vel_out);
    return CG_OK;
}

// ----------------------------------------------------------------------
// Batched binning phases (FP32 instances)
// ----------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) kb_bin_key(BLaunch L) {
    extern __shared__ int sh[];
    batch_loop(L, [&](const BInst& I, Blk b) {
        if (I.cellsort)
            bin_key_rank_body<float>(I.pos, I.n, I.gd, I.key, I.count, I.vol, I.status, nullptr, nullptr, nullptr,
                                     I.arrival, b);
        else
            bin_key_body<float>(I.pos, I.n, I.gd, I.key, I.count, I.hist, I.ntiles, I.b0, I.vol, I.status, sh, b);
    });
}

__global__ void __launch_bounds__(512) kb_bin_place(BLaunch L) {
    batch_loop(L, [&](const BInst& I, Blk b) { place_body(I.key, I.arrival, I.count, I.n, I.val1, b); });
}

__global__ void __launch_bounds__(kSegSortWarps * 32, 4) kb_seg_sort(BLaunch L) {
    batch_loop(L, [&](const BInst& I, Blk b) {
        seg_sort_body<float>(I.count, I.gd.nbulk, I.val1, I.key1, I.perm, I.key_sorted, I.inv_perm, I.vol,
                             I.vol_sorted, b);
    });
}

__global__ void __launch_bounds__(kSortThreads) kb_bin_hist1(BLaunch L) {
    extern __shared__ int sh[];
    batch_loop(L, [&](const BInst& I, Blk b) { bin_hist_body(I.key1, I.n, I.ntiles, I.b0, I.b1, I.hist, sh, b); });
}

__global__ void __launch_bounds__(kSortThreads, 2) kb_bin_scatter(BLaunch L, int pass) {
    extern __shared__ int cnt[];
    batch_loop(L, [&](const BInst& I, Blk b) {
        if (pass == 1)
            bin_scatter_body<false, true, float>(I.key1, I.val1, I.n, I.ntiles, I.b0, I.b1, I.hist, nullptr, nullptr,
                                                 I.perm, I.key_sorted, I.inv_perm, I.vol, I.vol_sorted, cnt, b);
        else if (I.npasses == 1)
            bin_scatter_body<true, true, float>(I.key, nullptr, I.n, I.ntiles, 0, I.b0, I.hist, nullptr, nullptr,
                                                I.perm, I.key_sorted, I.inv_perm, I.vol, I.vol_sorted, cnt, b);
        else
            bin_scatter_body<true, false, float>(I.key, nullptr, I.n, I.ntiles, 0, I.b0, I.hist, I.key1, I.val1,
                                                 nullptr, nullptr, nullptr, (const float*)nullptr, (float*)nullptr,
                                                 cnt, b);
    });
}

__global__ void __launch_bounds__(256) kb_scan_reduce(BLaunch L, int pass) {
    batch_loop(L, [&](const BInst& I, Blk b) { scan_reduce_body(pass ? I.scan1 : I.scan0, I.scan_part, b); });
}

__global__ void __launch_bounds__(256) kb_scan_down(BLaunch L, int pass) {
    batch_loop(L, [&](const BInst& I, Blk b) { scan_down_body(pass ? I.scan1 : I.scan0, I.scan_part, b); });
}

static PerDeviceOnce g_batch_attr_once;

static cg_status batch_bin_attrs() {
    return once_per_device(g_batch_attr_once, [] {
        const int mx = (int)scatter_smem_bytes(kMaxDigitBits, sizeof(float));
        CG_CUDA(cudaFuncSetAttribute(kb_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        CG_CUDA(cudaFuncSetAttribute(kb_bin_key, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (1 << kMaxDigitBits) * (int)sizeof(int)));
        CG_CUDA(cudaFuncSetAttribute(kb_bin_hist1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (1 << kMaxDigitBits) * (int)sizeof(int)));
        return CG_OK;
    });
}

cg_status launch_batch_bin(int phase, const BLaunch& L, unsigned grid, size_t smem, cudaStream_t s) {
    CG_TRY(batch_bin_attrs());
    if (L.total == 0 || grid == 0) return CG_OK;
    switch (phase) {
        case BP_KEY: kb_bin_key<<<grid, kSortThreads, smem, s>>>(L); break;
        case BP_SCAN0_R: kb_scan_reduce<<<grid, 256, 0, s>>>(L, 0); break;
        case BP_SCAN0_D: kb_scan_down<<<grid, 256, 0, s>>>(L, 0); break;
        case BP_SCAT0: kb_bin_scatter<<<grid, kSortThreads, smem, s>>>(L, 0); break;
        case BP_HIST1: kb_bin_hist1<<<grid, kSortThreads, smem, s>>>(L); break;
        case BP_SCAN1_R: kb_scan_reduce<<<grid, 256, 0, s>>>(L, 1); break;
        case BP_SCAN1_D: kb_scan_down<<<grid, 256, 0, s>>>(L, 1); break;
        case BP_SCAT1: kb_bin_scatter<<<grid, kSortThreads, smem, s>>>(L, 1); break;
        case BP_PLACE: kb_bin_place<<<grid, 512, 0, s>>>(L); break;
        case BP_SEGSORT: kb_seg_sort<<<grid, kSegSortWarps * 32, 0, s>>>(L); break;
        default: return CG_ERR_INVALID_ARG;
    }
    CG_CUDA(cudaGetLastError());
    return CG_OK;
}

int batch_bin_occupancy(int phase, size_t smem) {
    if (batch_bin_attrs() != CG_OK) return 1;
    int occ = 0;
    cudaError_t e = cudaSuccess;
    switch (phase) {
        case BP_KEY: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_bin_key, kSortThreads, smem); break;
        case BP_HIST1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_bin_hist1, kSortThreads, smem); break;
        case BP_SCAT0:
        case BP_SCAT1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_bin_scatter, kSortThreads, smem); break;
        case BP_SCAN0_R:
        case BP_SCAN1_R: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_scan_reduce, 256, 0); break;
        case BP_PLACE: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_bin_place, 512, 0); break;
        case BP_SEGSORT:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_seg_sort, kSegSortWarps * 32, 0);
            break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_scan_down, 256, 0); break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return occ > 0 ? occ : 1;
}

cg_status launch_bin(cg_grids* g, long long n, const void* pos_d, double* eps_fill, void* rec_fill,
                     void* eps_t_fill) {
    CG_TRY(set_attrs());
    const long long nbulk = g->gd.nbulk;
    // a binning of the same count held by the handle is the starting point
    // (rebin.cu), unless the descriptor asks for a digit sort
    const bool rebin = n > 0 && g->rb_rkn && g->hint_n == n && n <= g->cap &&
                       (g->desc.sort_digits == CG_SORT_AUTO || g->desc.sort_digits == CG_SORT_CELLS);
    const bool ident = rebin && pos_d == g->hint_ident;
    g->hint_n = -1;
    g->hint_ident = nullptr;
    g->n_binned = -1;
    g->vol_valid = false;
    g->key_valid = true;   // written by every path but the identity-hint rebinning
    if (rebin) {
        CG_TRY(launch_rebin(g, n, pos_d, ident, eps_fill, rec_fill, eps_t_fill));
        g->n_binned = n;
        g->vol_valid = true;
        g->key_valid = !ident;
        g->hint_n = n;
        return CG_OK;
    }
    // count[] lives in cell_start; the exclusive scan turns it into starts
    CG_CUDA(cudaMemsetAsync(g->cell_start, 0, sizeof(int32_t) * (nbulk + 1), g->stream));
    if (n == 0) {
        g->n_binned = 0;
        g->vol_valid = true;
        return CG_OK;
    }
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    const long long m0 = (long long)ntiles << g->pass_bits[0];
    if (use_cell_sort(g->desc.sort_digits, n, nbulk)) {
        if (g->fp64)
            CG_TRY(bin_rank<double>(g, n, (const double*)pos_d, ntiles, eps_fill, (double*)rec_fill,
                                    (double*)eps_t_fill));
        else
            CG_TRY(bin_rank<float>(g, n, (const float*)pos_d, ntiles, eps_fill, (float*)rec_fill,
                                   (float*)eps_t_fill));
        g->n_binned = n;
        g->vol_valid = true;
        g->hint_n = n;
        return CG_OK;
    }
    for (int p = 0; p < g->npasses; ++p)
        if (((long long)ntiles << g->pass_bits[p]) > g->hist_cap) return CG_ERR_OUT_OF_RANGE;

    if (g->fp64)
        CG_TRY(bin_passes<double>(g, n, (const double*)pos_d, ntiles, m0, eps_fill, (double*)rec_fill,
                                  (double*)eps_t_fill));
    else
        CG_TRY(bin_passes<float>(g, n, (const float*)pos_d, ntiles, m0, eps_fill, (float*)rec_fill,
                                 (float*)eps_t_fill));
    g->n_binned = n;
    g->vol_valid = true;
    g->hint_n = n;
    return CG_OK;
}

}  // namespace cg
