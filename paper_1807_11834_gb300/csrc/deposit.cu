// deposit.cu -- (a1) porosity and (a3) reaction deposition onto the bulk
// grid, the bulk pack feeding the drag gather, and the FP64 conservation
// sums.
//
// Porosity (Table 1 of arXiv 1807.11834: porosity field from the particle
// volumes of a cell; Sec. 2.4, beside Eq. DragLaw: porosity = fluid volume / cell volume):
// phi_B = sum_{p in B} V_p / V_B, eps_B = 1 - phi_B.
// Reaction (Eq. UFP: F_fpi is the fluid-side reaction to F_drag):
// S_B = -(1/V_B) sum_{p in B} F_p.
//
// Both are segmented sums over the stable bin order: one thread per bulk
// cell walks its segment in increasing particle index with a TwoSum
// compensated accumulator, so the result depends only on the particle set
// of the cell, never on the launch shape, and needs no atomics.  The
// porosity is formed in double from the compensated pair.
#include <algorithm>

#include "cg_internal.cuh"
#include "batch.cuh"

namespace cg {


// ----------------------------------------------------------------------
// Porosity over the sorted order (see seg_chunk_range): the segmented
// compensated sum of V_p leaves each cell's volume at its last slot, where
// eps = 1 - sum / V_B is formed in double.  Cells without particles are
// set to 1 beforehand by k_fill.
// ----------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void fill_body(T* __restrict__ a, long long m, T v, Blk b) {
    for (long long i = b.id * blockDim.x + threadIdx.x; i < m; i += b.n * blockDim.x) a[i] = v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_fill(T* __restrict__ a, long long m, T v) {
    pdl_wait();
    fill_body(a, m, v, launch_blk());
}

template <typename T>
__global__ void __launch_bounds__(256)
k_deposit_volume(const T* __restrict__ pos, long long n, const int32_t* __restrict__ perm,
                 const int32_t* __restrict__ key_sorted, const int32_t* __restrict__ cs, GridDev g,
                 double* __restrict__ eps, T* __restrict__ part, long long pstride, int do_sums) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    CSum<T> tot[1];
    for (long long base = wg * kSegChunk; base < n; base += nw * kSegChunk) {
        long long s, t;
        seg_chunk_range(base, n, key_sorted, cs, s, t);
        CSum<T> carry;
        int carry_key = -1;
        for (long long r = s; r < t; r += 32) {
            const long long i = r + lane;
            const bool valid = i < t;
            int key = -1;
            CSum<T> v[1];
            if (valid) {
                key = __ldg(key_sorted + i);
                const T d = __ldg(pos + 4 * (long long)__ldg(perm + i) + 3);
                sphere_volume_pair(d, v[0].s, v[0].c);
            }
            if (lane == 0 && key == carry_key) {
                CSum<T> c0 = carry;
                c0.merge(v[0]);
                v[0] = c0;
            }
            warp_seg_scan<T, 1>(v, key);
            int next = __shfl_down_sync(0xffffffffu, key, 1);
            if (lane == 31) next = (i + 1 < t) ? __ldg(key_sorted + i + 1) : -1;
            if (valid && next != key) {
                double e;
                T et;
                cell_porosity(v[0].s, v[0].c, g, e, et);
                eps[key] = e;
                tot[0].merge(v[0]);
            }
            carry.s = __shfl_sync(0xffffffffu, v[0].s, 31);
            carry.c = __shfl_sync(0xffffffffu, v[0].c, 31);
            carry_key = __shfl_sync(0xffffffffu, key, 31);
        }
    }
    if (do_sums) block_sums<T, 1>(tot, part, pstride, blockIdx.x);
}

// Porosity from the diameters already in sorted order (written by the final
// binning pass): each volume as an exact pair, compensated at every
// addition, so eps = 1 - phi keeps its accuracy in near-packed cells
// (phi -> 1) on the FP32 path.
template <typename T>
__device__ __forceinline__ void deposit_volume_sorted_body(const T* __restrict__ dsorted, long long n,
                                                           const int32_t* __restrict__ key_sorted,
                                                           const int32_t* __restrict__ cs, const GridDev& g,
                                                           double* __restrict__ eps, T* __restrict__ part,
                                                           long long pstride, int do_sums, Blk b,
                                                           T* __restrict__ rec = nullptr, T* __restrict__ eps_t = nullptr) {
    const long long wg = b.id * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = b.n * (blockDim.x >> 5);
    CSum<T> tot[1];
    for (long long base = wg * kSegChunk; base < n; base += nw * kSegChunk) {
        long long s, t;
        seg_chunk_range(base, n, key_sorted, cs, s, t);
        seg_seq<T, 1, true>(
            s, t, key_sorted,
            [&](long long i, CSum<T> (&v)[1]) { sphere_volume_pair(__ldg(dsorted + i), v[0].s, v[0].c); },
            [&](int key, const CSum<T> (&a)[1]) {
                double e;
                T et;
                cell_porosity(a[0].s, a[0].c, g, e, et);
                eps[key] = e;
                if (rec) rec[4 * (long long)key] = et;   // the drag record's porosity
                if (eps_t) eps_t[key] = et;
                tot[0].merge(a[0]);
            });
    }
    if (do_sums) block_sums<T, 1>(tot, part, pstride, b.id);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_deposit_volume_sorted(const T* __restrict__ dsorted, long long n, const int32_t* __restrict__ key_sorted,
                        const int32_t* __restrict__ cs, GridDev g, double* __restrict__ eps, T* __restrict__ part,
                        long long pstride, int do_sums, T* __restrict__ rec, T* __restrict__ eps_t) {
    pdl_wait();
    deposit_volume_sorted_body(dsorted, n, key_sorted, cs, g, eps, part, pstride, do_sums, launch_blk(), rec, eps_t);
}

// Reaction from the forces the drag wrote in sorted order (T4 per slot).
template <typename T>
__device__ __forceinline__ void deposit_sorted_force_body(const T* __restrict__ Fs, long long n,
                                                          const int32_t* __restrict__ key_sorted,
                                                          const int32_t* __restrict__ cs, const GridDev& g,
                                                          T* __restrict__ S, Blk b) {
    const long long wg = b.id * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = b.n * (blockDim.x >> 5);
    for (long long base = wg * kSegChunk; base < n; base += nw * kSegChunk) {
        long long s, t;
        seg_chunk_range(base, n, key_sorted, cs, s, t);
        seg_rounds<T, 3>(
            s, t, key_sorted,
            [&](long long i, T (&v)[3]) {
                const V4<T> f = ld4(Fs, i);
                v[0] = f.x;
                v[1] = f.y;
                v[2] = f.z;
            },
            [&](int key, CSum<T> (&a)[3]) { reaction_emit<T>(g, S, key, a); });
    }
}

// Semi-implicit coefficients (Eq. UFP): per cell A = (1/V_B) sum beta and
// b = (1/V_B) sum beta u_p from the drag's sorted (beta, beta u) records,
// with the reaction's segmented sums.
template <typename T>
__device__ __forceinline__ void deposit_implicit_body(const T* __restrict__ Bs, long long n,
                                                      const int32_t* __restrict__ key_sorted,
                                                      const int32_t* __restrict__ cs, const GridDev& g,
                                                      T* __restrict__ coef, Blk b) {
    const long long wg = b.id * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = b.n * (blockDim.x >> 5);
    for (long long base = wg * kSegChunk; base < n; base += nw * kSegChunk) {
        long long s, t;
        seg_chunk_range(base, n, key_sorted, cs, s, t);
        seg_rounds<T, 4>(
            s, t, key_sorted,
            [&](long long i, T (&v)[4]) {
                const V4<T> r = ld4(Bs, i);
                v[0] = r.x;
                v[1] = r.y;
                v[2] = r.z;
                v[3] = r.w;
            },
            [&](int key, CSum<T> (&a)[4]) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    coef[k * g.nbulk + key] = sizeof(T) == 4 ? a[k].get() * (T)g.invVBf : a[k].get() * (T)g.invVB;
            });
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_deposit_implicit(const T* __restrict__ Bs, long long n, const int32_t* __restrict__ key_sorted,
                   const int32_t* __restrict__ cs, GridDev g, T* __restrict__ coef) {
    pdl_wait();
    deposit_implicit_body<T>(Bs, n, key_sorted, cs, g, coef, launch_blk());
}

template <typename T>
__global__ void __launch_bounds__(256)
k_deposit_sorted_force(const T* __restrict__ Fs, long long n, const int32_t* __restrict__ key_sorted,
                       const int32_t* __restrict__ cs, GridDev g, T* __restrict__ S) {
    pdl_wait();
    deposit_sorted_force_body(Fs, n, key_sorted, cs, g, S, launch_blk());
}

// ----------------------------------------------------------------------
// Reaction source from caller-order SoA forces, over the sorted order as
// above (inside the coupling step the reaction is fused into the drag).
// S_B must be zero beforehand for cells without particles.
// ----------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_deposit_momentum(const T* __restrict__ F, long long n, const int32_t* __restrict__ perm,
                   const int32_t* __restrict__ key_sorted, const int32_t* __restrict__ cs, GridDev g,
                   T* __restrict__ S) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long base = wg * kSegChunk; base < n; base += nw * kSegChunk) {
        long long s, t;
        seg_chunk_range(base, n, key_sorted, cs, s, t);
        CSum<T> carry[3];
        int carry_key = -1;
        for (long long r = s; r < t; r += 32) {
            const long long i = r + lane;
            const bool valid = i < t;
            int key = -1;
            CSum<T> v[3];
            if (valid) {
                key = __ldg(key_sorted + i);
                const long long p = __ldg(perm + i);
                v[0].s = __ldg(F + p);
                v[1].s = __ldg(F + n + p);
                v[2].s = __ldg(F + 2 * n + p);
            }
            if (lane == 0 && key == carry_key)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    CSum<T> c0 = carry[k];
                    c0.merge(v[k]);
                    v[k] = c0;
                }
            warp_seg_scan<T, 3>(v, key);
            int next = __shfl_down_sync(0xffffffffu, key, 1);
            if (lane == 31) next = (i + 1 < t) ? __ldg(key_sorted + i + 1) : -1;
            if (valid && next != key)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    if (sizeof(T) == 4) S[k * g.nbulk + key] = -(v[k].get()) * (T)g.invVBf;
                    else S[k * g.nbulk + key] = -(v[k].get()) * (T)g.invVB;
                }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                carry[k].s = __shfl_sync(0xffffffffu, v[k].s, 31);
                carry[k].c = __shfl_sync(0xffffffffu, v[k].c, 31);
            }
            carry_key = __shfl_sync(0xffffffffu, key, 31);
        }
    }
}

// ----------------------------------------------------------------------
// Pack the bulk fields read by the drag gather: (eps, u_x, u_y, u_z) per
// cell in the path precision.  Interpolating eps itself (not 1 - eps) keeps
// the porosity at the particle accurate to a few roundings of eps also in
// near-packed cells, where the drag is most sensitive to it.
// ----------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void pack_body(const double* __restrict__ eps, const T* __restrict__ u, const GridDev& g,
                                          T* __restrict__ bulk4, T* __restrict__ eps_t, Blk b) {
    for (long long c = b.id * blockDim.x + threadIdx.x; c < g.nbulk; c += b.n * blockDim.x) {
        const double e = __ldg(eps + c);
        st4(bulk4, c, (T)e, __ldg(u + c), __ldg(u + g.nbulk + c), __ldg(u + 2 * g.nbulk + c));
        if (eps_t) eps_t[c] = (T)e;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_pack(const double* __restrict__ eps, const T* __restrict__ u, GridDev g, T* __restrict__ bulk4,
       T* __restrict__ eps_t) {
    pdl_wait();
    pack_body(eps, u, g, bulk4, eps_t, launch_blk());
}

// ----------------------------------------------------------------------
// Final FP64 reduction of the block partials (one block, fixed order)
// ----------------------------------------------------------------------

// One block per sum: merge the compensated pairs in a fixed order (strided
// per thread, then a fixed tree), convert the final pair to double.
template <typename T>
__device__ __forceinline__ void sums_body(const T* __restrict__ part, const SumsMap& map, double* __restrict__ sums,
                                          Blk b) {
    __shared__ T sh_s[8], sh_c[8];
    const int k = (int)b.id;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    CSum<T> a;
    if (map.off[k] >= 0)
        for (long long i = threadIdx.x; i < map.cnt[k]; i += blockDim.x) {
            CSum<T> o;
            o.s = part[2 * (map.off[k] + i)];
            o.c = part[2 * (map.off[k] + i) + 1];
            a.merge(o);
        }
    a = warp_reduce(a);
    if (lane == 0) {
        sh_s[warp] = a.s;
        sh_c[warp] = a.c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        CSum<T> t;
        t.s = sh_s[0];
        t.c = sh_c[0];
        for (int w = 1; w < 8; ++w) {
            CSum<T> o;
            o.s = sh_s[w];
            o.c = sh_c[w];
            t.merge(o);
        }
        sums[k] = map.off[k] >= 0 ? (double)t.s + (double)t.c : __longlong_as_double(0x7ff8000000000000LL);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sums(const T* __restrict__ part, SumsMap map, double* __restrict__ sums) {
    pdl_wait();
    sums_body(part, map, sums, launch_blk());
}

// ----------------------------------------------------------------------
// Batched phases (FP32 instances): zeroing, porosity, pack, reaction, sums
// ----------------------------------------------------------------------
// Cell counts to 0, porosity to 1 (cells without particles keep it), the
// reaction to 0 (cells without particles keep it).
__global__ void __launch_bounds__(256) kb_zero(BLaunch L) {
    batch_loop(L, [&](const BInst& I, Blk b) {
        fill_body<int32_t>(I.count, I.gd.nbulk + 1, 0, b);
        fill_body<double>(I.eps, I.gd.nbulk, 1.0, b);
        fill_body<float>(I.S_bulk, 3 * I.gd.nbulk, 0.f, b);
    });
}

__global__ void __launch_bounds__(256) kb_deposit_volume(BLaunch L) {
    batch_loop(L, [&](const BInst& I, Blk b) {
        deposit_volume_sorted_body<float>(I.vol_sorted, I.n, I.key_sorted, I.count, I.gd, I.eps,
                                          I.part + 2 * I.part_off[PS_VOL], I.part_blocks[PS_VOL], 1, b);
    });
}

__global__ void __launch_bounds__(256) kb_pack(BLaunch L) {
    batch_loop(L, [&](const BInst& I, Blk b) {
        pack_body<float>(I.eps, I.u_bulk, I.gd, I.bulk4, I.eps_fine ? I.eps_t : nullptr, b);
    });
}

__global__ void __launch_bounds__(256) kb_deposit_momentum(BLaunch L) {
    batch_loop(L, [&](const BInst& I, Blk b) {
        deposit_sorted_force_body<float>(I.Fs, I.n, I.key_sorted, I.count, I.gd, I.S_bulk, b);
    });
}

__global__ void __launch_bounds__(256) kb_sums(BLaunch L) {
    batch_loop(L, [&](const BInst& I, Blk b) { sums_body<float>(I.part, I.smap, I.sums, b); });
}

cg_status launch_batch_deposit(int phase, const BLaunch& L, unsigned grid, cudaStream_t s) {
    if (L.total == 0 || grid == 0) return CG_OK;
    switch (phase) {
        case BP_ZERO: kb_zero<<<grid, 256, 0, s>>>(L); break;
        case BP_DEPV: kb_deposit_volume<<<grid, 256, 0, s>>>(L); break;
        case BP_PACK: kb_pack<<<grid, 256, 0, s>>>(L); break;
        case BP_DEPM: kb_deposit_momentum<<<grid, 256, 0, s>>>(L); break;
        case BP_SUMS: kb_sums<<<grid, 256, 0, s>>>(L); break;
        default: return CG_ERR_INVALID_ARG;
    }
    CG_CUDA(cudaGetLastError());
    return CG_OK;
}

int batch_deposit_occupancy(int phase) {
    int occ = 0;
    cudaError_t e = cudaSuccess;
    switch (phase) {
        case BP_ZERO: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_zero, 256, 0); break;
        case BP_DEPV: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_deposit_volume, 256, 0); break;
        case BP_PACK: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_pack, 256, 0); break;
        case BP_DEPM: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_deposit_momentum, 256, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_sums, 256, 0); break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return occ > 0 ? occ : 1;
}

// ----------------------------------------------------------------------
// Launchers
// ----------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int per) { return (unsigned)((n + per - 1) / per); }

// Grid of the segmented deposits: at most one chunk per warp, and no more
// CTAs than are resident at once (4 per SM at their 64 registers), so the
// grid-stride loop runs without a second, partial wave.
static unsigned seg_blocks(cg_grids* g, long long n) {
    const long long chunks = (n + kSegChunk - 1) / kSegChunk;
    return (unsigned)std::max(1LL, std::min((chunks + 7) / 8, (long long)g->num_sms * 4));
}

cg_status launch_deposit_volume(cg_grids* g, long long n, const void* pos_d, double* eps, bool sums,
                                bool prefilled, void* rec, void* eps_t) {
    const unsigned fblk = (unsigned)std::min((g->gd.nbulk + 255) / 256, (long long)g->num_sms * 8);
    if (!prefilled || n == 0) CG_LAUNCH(g, "deposit_volume", k_fill<double>, fblk, 256, 0, eps, g->gd.nbulk, 1.0);
    const unsigned nblk = seg_blocks(g, n);
    void* part = part_ptr(g, PS_VOL);
    g->part_blocks[PS_VOL] = sums ? (long long)nblk : -1;
    if (sums && n == 0) {
        // no slots: the diagnostics partial is a single zero pair
        CG_CUDA(cudaMemsetAsync(part, 0, 2 * g->tsize, g->stream));
        g->part_blocks[PS_VOL] = 1;
        return CG_OK;
    }
    if (n == 0) return CG_OK;
    if (pos_d == nullptr) {
        // diameters already in sorted order from the binning of these positions
        if (g->fp64)
            CG_LAUNCH(g, "deposit_volume", k_deposit_volume_sorted<double>, nblk, 256, 0,
                      (const double*)g->vol_sorted, n, g->key_sorted, g->cell_start, g->gd, eps, (double*)part,
                      (long long)nblk, (int)sums, (double*)rec, (double*)eps_t);
        else
            CG_LAUNCH(g, "deposit_volume", k_deposit_volume_sorted<float>, nblk, 256, 0,
                      (const float*)g->vol_sorted, n, g->key_sorted, g->cell_start, g->gd, eps, (float*)part,
                      (long long)nblk, (int)sums, (float*)rec, (float*)eps_t);
        return CG_OK;
    }
    if (g->fp64)
        CG_LAUNCH(g, "deposit_volume", k_deposit_volume<double>, nblk, 256, 0, (const double*)pos_d, n, g->perm,
                  g->key_sorted, g->cell_start, g->gd, eps, (double*)part, (long long)nblk, (int)sums);
    else
        CG_LAUNCH(g, "deposit_volume", k_deposit_volume<float>, nblk, 256, 0, (const float*)pos_d, n, g->perm,
                  g->key_sorted, g->cell_start, g->gd, eps, (float*)part, (long long)nblk, (int)sums);
    return CG_OK;
}

cg_status launch_deposit_sorted_force(cg_grids* g, long long n, void* S_bulk) {
    CG_CUDA(cudaMemsetAsync(S_bulk, 0, 3 * g->tsize * (size_t)g->gd.nbulk, g->stream));
    if (n == 0) return CG_OK;
    const unsigned nblk = seg_blocks(g, n);
    if (g->fp64)
        CG_LAUNCH(g, "deposit_momentum", k_deposit_sorted_force<double>, nblk, 256, 0, (const double*)g->Fs, n,
                  g->key_sorted, g->cell_start, g->gd, (double*)S_bulk);
    else
        CG_LAUNCH(g, "deposit_momentum", k_deposit_sorted_force<float>, nblk, 256, 0, (const float*)g->Fs, n,
                  g->key_sorted, g->cell_start, g->gd, (float*)S_bulk);
    return CG_OK;
}

cg_status launch_deposit_implicit(cg_grids* g, long long n, void* coef_bulk) {
    CG_CUDA(cudaMemsetAsync(coef_bulk, 0, 4 * g->tsize * (size_t)g->gd.nbulk, g->stream));
    if (n == 0) return CG_OK;
    const unsigned nblk = seg_blocks(g, n);
    if (g->fp64)
        CG_LAUNCH(g, "deposit_implicit", k_deposit_implicit<double>, nblk, 256, 0, (const double*)g->Bs.p, n,
                  g->key_sorted, g->cell_start, g->gd, (double*)coef_bulk);
    else
        CG_LAUNCH(g, "deposit_implicit", k_deposit_implicit<float>, nblk, 256, 0, (const float*)g->Bs.p, n,
                  g->key_sorted, g->cell_start, g->gd, (float*)coef_bulk);
    return CG_OK;
}

cg_status launch_deposit_momentum(cg_grids* g, long long n, const void* force_soa, void* S_bulk) {
    CG_CUDA(cudaMemsetAsync(S_bulk, 0, 3 * g->tsize * (size_t)g->gd.nbulk, g->stream));
    if (n == 0) return CG_OK;
    const unsigned nblk = seg_blocks(g, n);
    if (g->fp64)
        CG_LAUNCH(g, "deposit_momentum", k_deposit_momentum<double>, nblk, 256, 0, (const double*)force_soa, n,
                  g->perm, g->key_sorted, g->cell_start, g->gd, (double*)S_bulk);
    else
        CG_LAUNCH(g, "deposit_momentum", k_deposit_momentum<float>, nblk, 256, 0, (const float*)force_soa, n,
                  g->perm, g->key_sorted, g->cell_start, g->gd, (float*)S_bulk);
    return CG_OK;
}

cg_status launch_pack(cg_grids* g, const double* eps, const void* u_bulk, bool want_eps_t) {
    const unsigned nblk = blocks_for(g->gd.nbulk, 256);
    if (g->fp64)
        CG_LAUNCH(g, "pack", k_pack<double>, nblk, 256, 0, eps, (const double*)u_bulk, g->gd,
                  (double*)g->bulk4, want_eps_t ? (double*)g->eps_t : nullptr);
    else
        CG_LAUNCH(g, "pack", k_pack<float>, nblk, 256, 0, eps, (const float*)u_bulk, g->gd, (float*)g->bulk4,
                  want_eps_t ? (float*)g->eps_t : nullptr);
    return CG_OK;
}

SumsMap sums_map(const long long* part_off, const long long* part_blocks) {
    SumsMap m;
    for (int k = 0; k < CG_NSUMS; ++k) {
        m.off[k] = -1;
        m.cnt[k] = 0;
    }
    auto col = [&](int dst, int region, int k) {
        if (part_blocks[region] >= 0) {
            m.off[dst] = part_off[region] + (long long)k * part_blocks[region];
            m.cnt[dst] = part_blocks[region];
        }
    };
    col(0, PS_DRAG, 0);
    col(1, PS_VOL, 0);
    for (int a = 0; a < 3; ++a) {
        col(2 + a, PS_DRAG, 1 + a);
        col(5 + a, PS_PROJ, 3 + a);   // S_B V_B: formed by the projection from the S_B it reads
        col(8 + a, PS_PROJ, a);
        col(12 + a, PS_DRAG, 5 + a);
    }
    col(11, PS_DRAG, 4);
    col(15, PS_DRAG, 8);
    return m;
}

cg_status launch_sums(cg_grids* g, double* sums) {
    const SumsMap m = sums_map(g->part_off, g->part_blocks);
    if (g->fp64)
        CG_LAUNCH(g, "sums", k_sums<double>, CG_NSUMS, 256, 0, (const double*)g->partials, m, sums);
    else
        CG_LAUNCH(g, "sums", k_sums<float>, CG_NSUMS, 256, 0, (const float*)g->partials, m, sums);
    return CG_OK;
}

}  // namespace cg
