// deposit.cu -- (a1) porosity and (a3) reaction deposition onto the bulk
// grid, the bulk pack feeding the drag gather, and the FP64 conservation
// sums.
//
// Porosity (Table 1 of arXiv 1807.11834: porosity field from the particle
// volumes of a cell; Sec. 2.3: porosity = fluid volume / cell volume):
// phi_B = sum_{p in B} V_p / V_B, eps_B = 1 - phi_B.
// Reaction (Eq. UFP: F_fpi is the counterpart of F_drag):
// S_B = -(1/V_B) sum_{p in B} F_p.
//
// Both are segmented sums over the stable bin order: one thread per bulk
// cell walks its segment in increasing particle index with a TwoSum
// compensated accumulator, so the result depends only on the particle set
// of the cell, never on the launch shape, and needs no atomics.  The
// porosity is formed in double from the compensated pair.
#include "cg_internal.cuh"

namespace cg {

template <typename T> __device__ __forceinline__ T pi_over_6();
template <> __device__ __forceinline__ float pi_over_6<float>() { return 0.52359877559829887f; }
template <> __device__ __forceinline__ double pi_over_6<double>() { return 0.52359877559829887308; }

// ----------------------------------------------------------------------
// Porosity: one warp per bulk cell, lanes strided over the cell's stable
// segment, compensated per-lane sums combined by a fixed xor tree.
// ----------------------------------------------------------------------
constexpr int kDepWarps = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kDepWarps)
k_deposit_volume(const T* __restrict__ pos, const int32_t* __restrict__ perm,
                 const int32_t* __restrict__ cs, GridDev g, double* __restrict__ eps,
                 T* __restrict__ part, long long pstride, int do_sums) {
    const int lane = threadIdx.x & 31;
    const long long c = (long long)blockIdx.x * kDepWarps + (threadIdx.x >> 5);
    CSum<T> cell_sum;
    if (c < g.nbulk) {
        const int b = __ldg(cs + c), e = __ldg(cs + c + 1);
        for (int i = b + lane; i < e; i += 32) {
            const T d = __ldg(pos + 4 * (long long)__ldg(perm + i) + 3);
            cell_sum.add(pi_over_6<T>() * d * d * d);
        }
        if (b != e) cell_sum = warp_reduce(cell_sum);
        if (lane == 0) eps[c] = 1.0 - ((double)cell_sum.s + (double)cell_sum.c) * g.invVB;
    }
    if (do_sums) {
        CSum<T> v[1];
        if (lane == 0) v[0] = cell_sum;
        block_sums<T, 1>(v, part, pstride);
    }
}

// ----------------------------------------------------------------------
// Reaction source from caller-order SoA forces, gathered through perm (one
// warp per cell as above).  Inside the coupling step the reaction is fused
// into the cell-order drag instead.
// ----------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(32 * kDepWarps)
k_deposit_momentum(const T* __restrict__ F, long long n, const int32_t* __restrict__ perm,
                   const int32_t* __restrict__ cs, GridDev g, T* __restrict__ S) {
    const int lane = threadIdx.x & 31;
    const long long c = (long long)blockIdx.x * kDepWarps + (threadIdx.x >> 5);
    if (c >= g.nbulk) return;
    CSum<T> a[3];
    const int b = __ldg(cs + c), e = __ldg(cs + c + 1);
    for (int i = b + lane; i < e; i += 32) {
        const long long p = __ldg(perm + i);
        a[0].add(__ldg(F + p));
        a[1].add(__ldg(F + n + p));
        a[2].add(__ldg(F + 2 * n + p));
    }
    if (b != e)
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] = warp_reduce(a[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (sizeof(T) == 4) S[k * g.nbulk + c] = -(a[k].get()) * (T)g.invVBf;
            else S[k * g.nbulk + c] = -(a[k].get()) * (T)g.invVB;
        }
}

// ----------------------------------------------------------------------
// Pack the bulk fields read by the drag gather: (phi, u_x, u_y, u_z) per
// cell in the path precision, phi = 1 - eps formed in double.
// ----------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_pack(const double* __restrict__ eps, const T* __restrict__ u, GridDev g, T* __restrict__ bulk4,
       T* __restrict__ eps_t) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.nbulk) return;
    const double e = __ldg(eps + c);
    st4(bulk4, c, (T)(1.0 - e), __ldg(u + c), __ldg(u + g.nbulk + c), __ldg(u + 2 * g.nbulk + c));
    if (eps_t) eps_t[c] = (T)e;
}

// ----------------------------------------------------------------------
// Final FP64 reduction of the block partials (one block, fixed order)
// ----------------------------------------------------------------------
struct SumsMap {
    long long off[CG_NSUMS];     // first pair of the partial column, -1 = not computed
    long long cnt[CG_NSUMS];     // number of partials
};

// One block per sum: merge the compensated pairs in a fixed order (strided
// per thread, then a fixed tree), convert the final pair to double.
template <typename T>
__global__ void __launch_bounds__(256) k_sums(const T* __restrict__ part, SumsMap map, double* __restrict__ sums) {
    __shared__ T sh_s[8], sh_c[8];
    const int k = blockIdx.x;
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

// ----------------------------------------------------------------------
// Launchers
// ----------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int per) { return (unsigned)((n + per - 1) / per); }

cg_status launch_deposit_volume(cg_grids* g, long long n, const void* pos_d, double* eps, bool sums) {
    (void)n;
    const unsigned nblk = blocks_for(g->gd.nbulk, kDepWarps);
    void* part = part_ptr(g, PS_VOL);
    g->part_blocks[PS_VOL] = sums ? (long long)nblk : -1;
    if (g->fp64)
        CG_LAUNCH(g, "deposit_volume", k_deposit_volume<double>, nblk, 32 * kDepWarps, 0, (const double*)pos_d, g->perm,
                  g->cell_start, g->gd, eps, (double*)part, (long long)nblk, (int)sums);
    else
        CG_LAUNCH(g, "deposit_volume", k_deposit_volume<float>, nblk, 32 * kDepWarps, 0, (const float*)pos_d, g->perm,
                  g->cell_start, g->gd, eps, (float*)part, (long long)nblk, (int)sums);
    return CG_OK;
}

cg_status launch_deposit_momentum(cg_grids* g, long long n, const void* force_soa, void* S_bulk) {
    const unsigned nblk = blocks_for(g->gd.nbulk, kDepWarps);
    if (g->fp64)
        CG_LAUNCH(g, "deposit_momentum", k_deposit_momentum<double>, nblk, 32 * kDepWarps, 0, (const double*)force_soa, n,
                  g->perm, g->cell_start, g->gd, (double*)S_bulk);
    else
        CG_LAUNCH(g, "deposit_momentum", k_deposit_momentum<float>, nblk, 32 * kDepWarps, 0, (const float*)force_soa, n,
                  g->perm, g->cell_start, g->gd, (float*)S_bulk);
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

cg_status launch_sums(cg_grids* g, double* sums) {
    SumsMap m;
    for (int k = 0; k < CG_NSUMS; ++k) {
        m.off[k] = -1;
        m.cnt[k] = 0;
    }
    auto col = [&](int dst, int region, int k) {
        if (g->part_blocks[region] >= 0) {
            m.off[dst] = g->part_off[region] + (long long)k * g->part_blocks[region];
            m.cnt[dst] = g->part_blocks[region];
        }
    };
    col(0, PS_DRAG, 0);
    col(1, PS_VOL, 0);
    for (int a = 0; a < 3; ++a) {
        col(2 + a, PS_DRAG, 1 + a);
        col(5 + a, PS_DRAG, kDragSums + a);
        col(8 + a, PS_PROJ, a);
        col(12 + a, PS_DRAG, 5 + a);
    }
    col(11, PS_DRAG, 4);
    col(15, PS_DRAG, 8);
    if (g->fp64)
        CG_LAUNCH(g, "sums", k_sums<double>, CG_NSUMS, 256, 0, (const double*)g->partials, m, sums);
    else
        CG_LAUNCH(g, "sums", k_sums<float>, CG_NSUMS, 256, 0, (const float*)g->partials, m, sums);
    return CG_OK;
}

}  // namespace cg
