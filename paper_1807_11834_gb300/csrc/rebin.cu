// rebin.cu -- incremental rebinning: the per-step particle-to-cell
// connectivity rebuild of Sec. 2.2 of arXiv 1807.11834, started from the
// binning of the previous step.
//
// From one coupling step to the next a particle moves a small fraction of a
// bulk cell, so most particles keep their cell.  The handle's last binning
// of the same particle count (perm_old, key_sorted_old, cell_start_old: the
// stable order, ids ascending within each cell) is therefore nearly the
// new one.  Call a particle whose cell is unchanged a stayer and one whose
// cell changed a mover.  Stayers keep their relative order (their old order
// is sorted by (cell, id) and their cells did not change), so with
//   D(s)   = movers at old slots before s (departures),
//   A(c)   = movers arriving in cells before c,
//   a_c(i) = movers arriving in c with an id below i,
// the new slot of the stayer at old slot s, of cell c and id i, is
//   s - D(s) + A(c) + a_c(i),
// and the new slot of a mover i arriving in c is
//   start_new(c) + (stayers of c with an id below i) + a_c(i),
// where start_new is the exclusive scan of the new counts
// count_old(c) - departures(c) + arrivals(c).  This holds for any new
// positions and any valid binning of the same count: the old order only
// decides how many particles are movers, never the result, which is the
// stable order of the new cells exactly as a full sort gives it.
//
// Old slot s holds particle perm_old[s] when the caller kept its particle
// order, or particle s when the particles are the sorted output of the last
// step (cg_step_sorted; the identity hint).  When a cell receives more than
// kRebinMaxArrivals movers (the movers' searches and counts grow with the
// arrivals of their cell) the device falls back to the per-cell sort: both
// paths are launched and
// each kernel checks a device flag, so a captured CUDA graph takes the
// right path on every replay.  The same holds when no particle changed its
// cell: the scans return at once on a device count of the movers, and the
// kernels after them keep the old bins.
#include <algorithm>

#include "cg_internal.cuh"

namespace cg {

namespace {

enum { RB_FALLBACK = 0, RB_MOVERS = 1 };   // counters: fallback flag, movers
constexpr int kCellBits = 22;   // a mover entry packs its new cell (< 2^22) and arrival rank (< 2^8)

struct RebinPtrs {
    int32_t* cnt;       // [n_b + 1] new counts, then (scanned in place) new starts
    int32_t* arr;       // [n_b + 1] arrivals per cell, then their starts
    int32_t* dep;       // [n_b + 1] departures per cell
    int32_t* blk;       // [nblk + 1] departures per block of old slots, then their starts
    int32_t* ctr;       // [kRebinCounters] movers, fallback flag
};

RebinPtrs rebin_ptrs(cg_grids* g) {
    const long long nb1 = rebin_pad(g->gd.nbulk + 1);
    RebinPtrs r;
    r.cnt = g->rb_small;
    r.arr = r.cnt + nb1;
    r.dep = r.arr + nb1;
    r.blk = r.dep + nb1;
    r.ctr = r.blk + rebin_pad(g->rb_nblk + 1);
    return r;
}

// Set every cell's porosity to 1 (and that of the drag record and of its
// path-precision copy); the porosity deposit overwrites the occupied cells.
template <typename T>
__device__ __forceinline__ void eps_fill_cells(long long nbulk, double* __restrict__ eps_fill,
                                               T* __restrict__ rec_fill, T* __restrict__ eps_t_fill) {
    if (!eps_fill) return;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nbulk;
         c += (long long)gridDim.x * blockDim.x) {
        eps_fill[c] = 1.0;
        if (rec_fill) rec_fill[4 * c] = T(1);
        if (eps_t_fill) eps_t_fill[c] = T(1);
    }
}

__device__ __forceinline__ void add_status_counts(unsigned long long* st, int outside, int nonfin) {
    if (outside) {
        atomicAdd(&st[ST_OUTSIDE], (unsigned long long)outside);
        atomicOr(&st[ST_FLAGS], (unsigned long long)CG_FLAG_OUTSIDE);
    }
    if (nonfin) {
        atomicAdd(&st[ST_NONFINITE], (unsigned long long)nonfin);
        atomicOr(&st[ST_FLAGS], (unsigned long long)CG_FLAG_NONFINITE);
    }
}

// Cell and diameter of particle p (caller order, record v), with the status counts.
template <typename T>
__device__ __forceinline__ int key_of(const V4<T>& v, long long p, const GridDev& g, int32_t* __restrict__ key,
                                      T* __restrict__ vol, int& n_out, int& n_nf) {
    int outside = 0;
    if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) n_nf++;
    const int c = cell_of(v, g, outside);
    n_out += outside;
    key[p] = c;
    vol[p] = v.w;   // the diameter: the porosity forms the volume as an exact pair
    return c;
}

__device__ __forceinline__ void flush_status(unsigned long long* st, int n_out, int n_nf) {
    n_out = __reduce_add_sync(0xffffffffu, n_out);
    n_nf = __reduce_add_sync(0xffffffffu, n_nf);
    if ((threadIdx.x & 31) == 0 && (n_out | n_nf)) add_status_counts(st, n_out, n_nf);
}

}  // namespace

// Cells and diameters in the caller's order (the particles kept their order:
// old slot s holds perm_old[s]).  FP32: six CTAs per SM (40 registers),
// the loads of more warps in flight (measured faster than four).
template <typename T>
__global__ void __launch_bounds__(kRebinThreads, sizeof(T) == 4 ? 6 : 4)
k_rebin_key(const T* __restrict__ pos, long long n, GridDev g, int32_t* __restrict__ key, T* __restrict__ vol,
            unsigned long long* __restrict__ status, double* __restrict__ eps_fill, T* __restrict__ rec_fill,
            T* __restrict__ eps_t_fill) {
    pdl_wait();
    int n_out = 0, n_nf = 0;
    const long long base = (long long)blockIdx.x * kRebinTile;
    V4<T> pv[kRebinItems];
    // every load of the thread first, so that they are in flight together
#pragma unroll
    for (int k = 0; k < kRebinItems; ++k) {
        const long long p = base + k * kRebinThreads + threadIdx.x;
        if (p < n) pv[k] = ld4(pos, p);
    }
#pragma unroll
    for (int k = 0; k < kRebinItems; ++k) {
        const long long p = base + k * kRebinThreads + threadIdx.x;
        if (p < n) key_of(pv[k], p, g, key, vol, n_out, n_nf);
    }
    flush_status(status, n_out, n_nf);
    eps_fill_cells<T>(g.nbulk, eps_fill, rec_fill, eps_t_fill);
}

// Mark the movers, over the old slots (slot base + k * threads + t of
// thread t, so every load and store of a row is coalesced): the new cell of
// every old slot, complemented for a mover (rkn), and the old id (rid, only
// when the particles kept the caller's order); per mover one departure
// from its old cell, one arrival (with its rank) in its new cell and an
// entry in the block's own part of the mover list (kRebinTile entries per
// block: no atomic decides a position); the movers of each block.  IDENT: old slot s holds particle
// s, whose cell and diameter are formed here.
template <typename T, bool IDENT>
__global__ void __launch_bounds__(kRebinThreads)
k_rebin_mark(const T* __restrict__ pos, long long n, GridDev g, const int32_t* __restrict__ perm_old,
             const int32_t* __restrict__ ks_old, int32_t* __restrict__ key, T* __restrict__ vol,
             int32_t* __restrict__ rid, int32_t* __restrict__ rkn, int32_t* __restrict__ arr,
             int32_t* __restrict__ dep, int2* __restrict__ mov, int32_t* __restrict__ blk_dep,
             int32_t* __restrict__ ctr, unsigned long long* __restrict__ status, double* __restrict__ eps_fill,
             T* __restrict__ rec_fill, T* __restrict__ eps_t_fill) {
    pdl_wait();
    constexpr int W = kRebinThreads / 32;
    __shared__ int s_cnt[W];
    __shared__ int s_base[W];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kRebinTile;
    int n_out = 0, n_nf = 0;
    int idk[kRebinItems], cnk[kRebinItems], cok[kRebinItems];
    V4<T> pv[kRebinItems];
    // every load of the thread first, so that they are in flight together
#pragma unroll
    for (int k = 0; k < kRebinItems; ++k) {
        const long long s = base + k * kRebinThreads + threadIdx.x;
        idk[k] = -1;
        cnk[k] = cok[k] = 0;
        if (s < n) {
            idk[k] = IDENT ? (int)s : __ldg(perm_old + s);
            cok[k] = __ldg(ks_old + s);
            if (IDENT) pv[k] = ld4(pos, s);
        }
    }
#pragma unroll
    for (int k = 0; k < kRebinItems; ++k) {
        const long long s = base + k * kRebinThreads + threadIdx.x;
        if (s >= n) continue;
        if (IDENT) {
            // the cell itself is kept only in rkn below (key is formed from it on demand)
            int outside = 0;
            const V4<T>& v = pv[k];
            if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) n_nf++;
            cnk[k] = cell_of(v, g, outside);
            n_out += outside;
            vol[s] = v.w;   // the diameter: the porosity forms the volume as an exact pair
        } else {
            cnk[k] = __ldg(key + idk[k]);
        }
    }
    unsigned mb[kRebinItems];
    int wc = 0;
#pragma unroll
    for (int k = 0; k < kRebinItems; ++k) {
        const long long s = base + k * kRebinThreads + threadIdx.x;
        const bool valid = s < n;
        const bool moved = valid && cnk[k] != cok[k];
        mb[k] = __ballot_sync(full, moved);
        wc += __popc(mb[k]);
        if (valid) {
            rkn[s] = moved ? ~cnk[k] : cnk[k];
            if (!IDENT) rid[s] = idk[k];
        }
    }
    if (lane == 0) s_cnt[warp] = wc;
    if (IDENT) flush_status(status, n_out, n_nf);
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            s_base[w] = t;
            t += s_cnt[w];
        }
        blk_dep[blockIdx.x] = t;
        if (t) atomicAdd(&ctr[RB_MOVERS], t);
    }
    __syncthreads();
    if (wc) {
        long long idx = base + s_base[warp];
#pragma unroll
        for (int k = 0; k < kRebinItems; ++k) {
            if (mb[k] >> lane & 1u) {
                const long long j = idx + __popc(mb[k] & lanemask_lt());
                atomicAdd(&dep[cok[k]], 1);
                const int r = atomicAdd(&arr[cnk[k]], 1);
                if (r < kRebinMaxArrivals) mov[j] = make_int2(idk[k], cnk[k] | (r << kCellBits));
                else ctr[RB_FALLBACK] = 1;
            }
            idx += __popc(mb[k]);
        }
    }
    if (IDENT) eps_fill_cells<T>(g.nbulk, eps_fill, rec_fill, eps_t_fill);
}

// The new count of every cell (the new starts themselves when no particle
// changed its cell: the scans are then left out); or, when the device falls back to the
// per-cell sort, that sort's per-cell counts and arrival ranks (consecutive
// lanes on consecutive particles, one atomic per run of equal cells), from
// the cells already formed (IDENT: from rkn, whose cells are written to key
// here for the sort's placement).
template <bool IDENT>
__global__ void __launch_bounds__(kRebinThreads)
k_rebin_cells(const int32_t* __restrict__ cs_old, long long nbulk, const int32_t* __restrict__ dep,
              const int32_t* __restrict__ arr, int32_t* __restrict__ cnt, const int32_t* __restrict__ ctr,
              int32_t* __restrict__ key, const int32_t* __restrict__ rkn, long long n, int32_t* __restrict__ arrival) {
    pdl_wait();
    if (!ctr[RB_FALLBACK]) {
        if (ctr[RB_MOVERS] == 0) {
            // no particle changed its cell: the new starts are the old ones,
            // written in their scanned form (the scans are left out; the
            // arrivals and departures, all zero, are their own scans)
            for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c <= nbulk;
                 c += (long long)gridDim.x * blockDim.x)
                cnt[c] = __ldg(cs_old + c);
            return;
        }
        for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nbulk;
             c += (long long)gridDim.x * blockDim.x)
            cnt[c] = __ldg(cs_old + c + 1) - __ldg(cs_old + c) - __ldg(dep + c) + __ldg(arr + c);
        return;
    }
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * kRebinTile; base < n; base += (long long)gridDim.x * kRebinTile) {
        int ck[kRebinItems], lk[kRebinItems], old[kRebinItems];
#pragma unroll
        for (int k = 0; k < kRebinItems; ++k) {
            const long long p = base + k * kRebinThreads + threadIdx.x;
            const bool valid = p < n;
            ck[k] = -1;
            if (valid) {
                if (IDENT) {
                    const int r = __ldg(rkn + p);
                    ck[k] = r >= 0 ? r : ~r;
                    key[p] = ck[k];
                } else {
                    ck[k] = __ldg(key + p);
                }
            }
            lk[k] = run_head_length(ck[k], valid);
        }
#pragma unroll
        for (int k = 0; k < kRebinItems; ++k) old[k] = lk[k] ? atomicAdd(&cnt[ck[k]], lk[k]) : 0;
#pragma unroll
        for (int k = 0; k < kRebinItems; ++k) {
            const long long p = base + k * kRebinThreads + threadIdx.x;
            const unsigned heads = __ballot_sync(full, lk[k] != 0);
            const int head = 31 - __clz(heads & ((2u << lane) - 1u));
            const int o = __shfl_sync(full, old[k], head < 0 ? 0 : head);
            if (p < n) arrival[p] = o + lane - head;
        }
    }
}

// The caller-order cells of an identity-hint binning, from the records
// (a caller asks for them, or the handle needs them).
__global__ void __launch_bounds__(256) k_rebin_keys(const int32_t* __restrict__ rkn, long long n,
                                                    int32_t* __restrict__ key) {
    pdl_wait();
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int r = __ldg(rkn + p);
        key[p] = r >= 0 ? r : ~r;
    }
}

// Each mover into the arrival list of its new cell, at its arrival rank:
// one warp per block of old slots walks that block's movers.
__global__ void __launch_bounds__(256)
k_rebin_place(const int2* __restrict__ mov, const int32_t* __restrict__ blk_start, long long nblk,
              const int32_t* __restrict__ arr_start, int2* __restrict__ arr_list, const int32_t* __restrict__ ctr) {
    pdl_wait();
    if (ctr[RB_FALLBACK]) return;
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nblk; b += nw) {
        const int cnt = __ldg(blk_start + b + 1) - __ldg(blk_start + b);
        for (int j = lane; j < cnt; j += 32) {
            const int2 m = mov[b * kRebinTile + j];
            const int c = m.y & ((1 << kCellBits) - 1), r = m.y >> kCellBits;
            arr_list[__ldg(arr_start + c) + r] = make_int2(m.x, c);
        }
    }
}

// Arrivals in the list [a0, a1) with an id below i.
__device__ __forceinline__ int arrivals_below(const int2* __restrict__ arr_list, int a0, int a1, int i) {
    int a = 0;
    for (int q = a0; q < a1; ++q) a += __ldg(&arr_list[q].x) < i;
    return a;
}

template <typename T>
__device__ __forceinline__ void emit(long long n, long long ns, int i, int c, int32_t* __restrict__ perm,
                                     int32_t* __restrict__ key_sorted, int32_t* __restrict__ inv_perm,
                                     const T* __restrict__ vol, T* __restrict__ vol_sorted) {
    if ((unsigned long long)ns >= (unsigned long long)n) return;   // never for a valid binning
    perm[ns] = i;
    key_sorted[ns] = c;
    inv_perm[i] = (int)ns;
    vol_sorted[ns] = __ldg(vol + i);
}

// Stayers, over the old slots in the layout of the mark kernel (coalesced
// rows).  Departures before a slot: the block's start (scan of the block
// totals), the rows and warps before it in the block (a table of warp
// counts), and the lanes before it (ballot).
template <typename T, bool IDENT>
__device__ __forceinline__ void rebin_stay_body(const int32_t* __restrict__ rid, const int32_t* __restrict__ rkn,
                                                long long n, const int32_t* __restrict__ blk_start,
                                                const int32_t* __restrict__ arr_start, const int2* __restrict__ arr_list,
                                                const T* __restrict__ vol, int32_t* __restrict__ perm,
                                                int32_t* __restrict__ key_sorted, int32_t* __restrict__ inv_perm,
                                                T* __restrict__ vol_sorted, long long bid, long long nblk) {
    const long long base0 = bid * kRebinTile;
    if (__ldg(blk_start + nblk) == 0) {
        // no particle changed its cell (the scanned departures sum to zero):
        // slot s keeps its particle and cell, so key_sorted stands, and in the
        // caller's order perm and inv_perm stand too; the diameters are read
        // afresh (a particle may have changed its size)
        int ik[kRebinItems];
        T dk[kRebinItems];
#pragma unroll
        for (int k = 0; k < kRebinItems; ++k) {
            const long long s = base0 + k * kRebinThreads + threadIdx.x;
            ik[k] = IDENT ? (int)s : (s < n ? __ldg(rid + s) : 0);
        }
#pragma unroll
        for (int k = 0; k < kRebinItems; ++k) {
            const long long s = base0 + k * kRebinThreads + threadIdx.x;
            if (s < n) dk[k] = __ldg(vol + ik[k]);
        }
#pragma unroll
        for (int k = 0; k < kRebinItems; ++k) {
            const long long s = base0 + k * kRebinThreads + threadIdx.x;
            if (s >= n) continue;
            vol_sorted[s] = dk[k];
            if (IDENT) {
                perm[s] = ik[k];
                inv_perm[ik[k]] = (int)s;
            }
        }
        return;
    }
    constexpr int W = kRebinThreads / 32;
    __shared__ int s_tab[kRebinItems * W];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = base0;
    int kn[kRebinItems], id[kRebinItems], a0[kRebinItems], a1[kRebinItems];
    T d[kRebinItems];
    unsigned db[kRebinItems];
#pragma unroll
    for (int k = 0; k < kRebinItems; ++k) {
        const long long s = base + k * kRebinThreads + threadIdx.x;
        kn[k] = s < n ? __ldg(rkn + s) : -1;
        id[k] = IDENT ? (int)s : (s < n ? __ldg(rid + s) : 0);
    }
    // the gathers of each stayer (its cell's arrivals, its diameter) go out
    // before the block waits for the departure table
#pragma unroll
    for (int k = 0; k < kRebinItems; ++k) {
        const long long s = base + k * kRebinThreads + threadIdx.x;
        a0[k] = a1[k] = 0;
        if (s < n && kn[k] >= 0) {
            a0[k] = __ldg(arr_start + kn[k]);
            a1[k] = __ldg(arr_start + kn[k] + 1);
            d[k] = __ldg(vol + id[k]);
        }
        db[k] = __ballot_sync(full, s < n && kn[k] < 0);
        if (lane == 0) s_tab[k * W + warp] = __popc(db[k]);
    }
    __syncthreads();
    static_assert(kRebinItems * W == 32, "one lane per (row, warp) entry");
    if (warp == 0) {   // exclusive prefix over (row, warp) in slot order: one shuffle scan
        const int c = s_tab[lane];
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(full, incl, off);
            if (lane >= off) incl += o;
        }
        s_tab[lane] = __ldg(blk_start + bid) + incl - c;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRebinItems; ++k) {
        const long long s = base + k * kRebinThreads + threadIdx.x;
        if (s >= n || kn[k] < 0) continue;
        const int D = s_tab[k * W + warp] + __popc(db[k] & lanemask_lt());
        const int c = kn[k], i = id[k];
        const long long ns = s - D + a0[k] + (a1[k] > a0[k] ? arrivals_below(arr_list, a0[k], a1[k], i) : 0);
        if ((unsigned long long)ns >= (unsigned long long)n) continue;   // never for a valid binning
        perm[ns] = i;
        key_sorted[ns] = c;
        inv_perm[i] = (int)ns;
        vol_sorted[ns] = d[k];
    }
}

// Movers: the stayers of the new cell with an id below the mover's (a binary
// search over the old segment, whose ids ascend, then a count of the
// stayers before that point) and the arrivals with an id below it.
template <typename T, bool IDENT>
__device__ __forceinline__ void rebin_movers_body(const int32_t* __restrict__ rid, const int32_t* __restrict__ rkn,
                                                  long long n, const int32_t* __restrict__ cs_old,
                                                  const int32_t* __restrict__ cs_new,
                                                  const int32_t* __restrict__ arr_start,
                                                  const int2* __restrict__ arr_list, long long nbulk,
                                                  const T* __restrict__ vol, int32_t* __restrict__ perm,
                                                  int32_t* __restrict__ key_sorted, int32_t* __restrict__ inv_perm,
                                                  T* __restrict__ vol_sorted, long long bid, long long nb) {
    const long long nm = __ldg(arr_start + nbulk);   // all arrivals
    for (long long q = bid * blockDim.x + threadIdx.x; q < nm; q += nb * blockDim.x) {
        const int2 m = arr_list[q];
        const int i = m.x, c = m.y;
        const int o0 = __ldg(cs_old + c), o1 = __ldg(cs_old + c + 1);
        int lo = o0, hi = o1;
        if (IDENT) {
            lo = i < o0 ? o0 : (i > o1 ? o1 : i);   // the old ids of the segment are its slots
        } else {
            while (lo < hi) {
                const int mid = lo + ((hi - lo) >> 1);
                if (__ldg(rid + mid) < i) lo = mid + 1;
                else hi = mid;
            }
        }
        int stay = 0;
        for (int p = o0; p < lo; ++p) stay += __ldg(rkn + p) >= 0;
        const int a0 = __ldg(arr_start + c), a1 = __ldg(arr_start + c + 1);
        const long long ns = (long long)__ldg(cs_new + c) + stay + arrivals_below(arr_list, a0, a1, i);
        emit<T>(n, ns, i, c, perm, key_sorted, inv_perm, vol, vol_sorted);
    }
}

// Every particle's new slot in one launch: blocks [0, mgrid) place the
// movers (first, so that their searches run beside the stayers), blocks
// [mgrid, mgrid + nblk) the stayers of one block of old slots each.
template <typename T, bool IDENT>
__global__ void __launch_bounds__(kRebinThreads)
k_rebin_slots(const int32_t* __restrict__ rid, const int32_t* __restrict__ rkn, long long n,
              const int32_t* __restrict__ blk_start, const int32_t* __restrict__ cs_old,
              const int32_t* __restrict__ cs_new, const int32_t* __restrict__ arr_start,
              const int2* __restrict__ arr_list, long long nbulk, const T* __restrict__ vol,
              int32_t* __restrict__ perm, int32_t* __restrict__ key_sorted, int32_t* __restrict__ inv_perm,
              T* __restrict__ vol_sorted, const int32_t* __restrict__ ctr, long long nblk, long long mgrid) {
    pdl_wait();
    if (ctr[RB_FALLBACK]) return;
    if ((long long)blockIdx.x < mgrid)
        rebin_movers_body<T, IDENT>(rid, rkn, n, cs_old, cs_new, arr_start, arr_list, nbulk, vol, perm, key_sorted,
                                    inv_perm, vol_sorted, blockIdx.x, mgrid);
    else
        rebin_stay_body<T, IDENT>(rid, rkn, n, blk_start, arr_start, arr_list, vol, perm, key_sorted, inv_perm,
                                  vol_sorted, blockIdx.x - mgrid, nblk);
}

template <typename T>
static cg_status rebin_impl(cg_grids* g, long long n, const T* pos, bool ident, double* eps_fill, T* rec_fill,
                            T* eps_t_fill) {
    const long long nbulk = g->gd.nbulk;
    const RebinPtrs R = rebin_ptrs(g);
    const long long nblk = (n + kRebinTile - 1) / kRebinTile;
    if (nblk > g->rb_nblk) return CG_ERR_OUT_OF_RANGE;
    CG_CUDA(cudaMemsetAsync(g->rb_small, 0, sizeof(int32_t) * rebin_small_ints(nbulk, g->rb_nblk), g->stream));
    if (!ident)
        CG_LAUNCH(g, "rebin_key", k_rebin_key<T>, (unsigned)nblk, kRebinThreads, 0, pos, n, g->gd, g->key, (T*)g->vol,
                  g->status, eps_fill, rec_fill, eps_t_fill);
    if (ident)
        CG_LAUNCH(g, "rebin_mark", (k_rebin_mark<T, true>), (unsigned)nblk, kRebinThreads, 0, pos, n, g->gd,
                  (const int32_t*)nullptr, (const int32_t*)g->key_sorted, g->key, (T*)g->vol, g->rb_rid, g->rb_rkn,
                  R.arr, R.dep, g->rb_mov, R.blk, R.ctr, g->status, eps_fill, rec_fill, eps_t_fill);
    else
        CG_LAUNCH(g, "rebin_mark", (k_rebin_mark<T, false>), (unsigned)nblk, kRebinThreads, 0, pos, n, g->gd,
                  (const int32_t*)g->perm, (const int32_t*)g->key_sorted, g->key, (T*)g->vol, g->rb_rid, g->rb_rkn,
                  R.arr, R.dep, g->rb_mov, R.blk, R.ctr, g->status, (double*)nullptr, (T*)nullptr, (T*)nullptr);
    const unsigned cgrid = (unsigned)std::max<long long>(1, std::min<long long>(std::max((nbulk + 255) / 256, nblk),
                                                                               (long long)g->num_sms * 8));
    if (ident)
        CG_LAUNCH(g, "rebin_cells", k_rebin_cells<true>, cgrid, kRebinThreads, 0, (const int32_t*)g->cell_start,
                  nbulk, (const int32_t*)R.dep, (const int32_t*)R.arr, R.cnt, (const int32_t*)R.ctr, g->key,
                  (const int32_t*)g->rb_rkn, n, g->key2);
    else
        CG_LAUNCH(g, "rebin_cells", k_rebin_cells<false>, cgrid, kRebinThreads, 0, (const int32_t*)g->cell_start,
                  nbulk, (const int32_t*)R.dep, (const int32_t*)R.arr, R.cnt, (const int32_t*)R.ctr, g->key,
                  (const int32_t*)g->rb_rkn, n, g->key2);
    {
        const int32_t* in[3] = {R.cnt, R.arr, R.blk};
        int32_t* out[3] = {R.cnt, R.arr, R.blk};
        const long long m[3] = {nbulk + 1, nbulk + 1, nblk + 1};
        CG_TRY(scan_exclusive(g, 3, in, out, m, R.ctr + RB_MOVERS));
    }
    const unsigned pgrid = (unsigned)std::max<long long>(1, std::min<long long>((nblk + 7) / 8, (long long)g->num_sms * 8));
    CG_LAUNCH(g, "rebin_place", k_rebin_place, pgrid, 256, 0, (const int2*)g->rb_mov, (const int32_t*)R.blk, nblk,
              (const int32_t*)R.arr, g->rb_arr, (const int32_t*)R.ctr);
    const long long mgrid = (long long)g->num_sms * 8;
#define CG_REBIN_SLOTS(ID)                                                                                        \
    CG_LAUNCH(g, "rebin_slots", (k_rebin_slots<T, ID>), (unsigned)(mgrid + nblk), kRebinThreads, 0,                 \
              (const int32_t*)g->rb_rid, (const int32_t*)g->rb_rkn, n, (const int32_t*)R.blk,                      \
              (const int32_t*)g->cell_start, (const int32_t*)R.cnt, (const int32_t*)R.arr, (const int2*)g->rb_arr,   \
              nbulk, (const T*)g->vol, g->perm, g->key_sorted, g->inv_perm, (T*)g->vol_sorted,                      \
              (const int32_t*)R.ctr, nblk, mgrid)
    if (ident) {
        CG_REBIN_SLOTS(true);
    } else {
        CG_REBIN_SLOTS(false);
    }
#undef CG_REBIN_SLOTS
    // fallback: placement and per-cell sort from the scanned counts
    CG_TRY(launch_cellsort_tail(g, n, R.cnt, R.ctr + RB_FALLBACK));
    CG_CUDA(cudaMemcpyAsync(g->cell_start, R.cnt, sizeof(int32_t) * (nbulk + 1), cudaMemcpyDeviceToDevice, g->stream));
    return CG_OK;
}

// The caller-order cells of the last binning (g->key), formed from the
// mover records when an identity-hint binning left them out.
cg_status ensure_keys(cg_grids* g, long long n) {
    if (g->key_valid || n <= 0) return CG_OK;
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, (long long)g->num_sms * 8);
    CG_LAUNCH(g, "rebin_keys", k_rebin_keys, grid, 256, 0, (const int32_t*)g->rb_rkn, n, g->key);
    g->key_valid = true;
    return CG_OK;
}

cg_status launch_rebin(cg_grids* g, long long n, const void* pos_d, bool ident, double* eps_fill, void* rec_fill,
                       void* eps_t_fill) {
    if (g->fp64) return rebin_impl<double>(g, n, (const double*)pos_d, ident, eps_fill, (double*)rec_fill,
                                           (double*)eps_t_fill);
    return rebin_impl<float>(g, n, (const float*)pos_d, ident, eps_fill, (float*)rec_fill, (float*)eps_t_fill);
}

}  // namespace cg
