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
// Porosity
// ----------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_deposit_volume(const T* __restrict__ pos, const int32_t* __restrict__ perm,
                 const int32_t* __restrict__ cs, GridDev g, double* __restrict__ eps,
                 double* __restrict__ part, long long pstride, int do_sums) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    CSum<T> cell_sum;
    if (c < g.nbulk) {
        const int b = __ldg(cs + c), e = __ldg(cs + c + 1);
        int i = b;
        // 4-way unrolled gather to keep several loads in flight
        for (; i + 4 <= e; i += 4) {
            int p0 = __ldg(perm + i), p1 = __ldg(perm + i + 1), p2 = __ldg(perm + i + 2), p3 = __ldg(perm + i + 3);
            T d0 = __ldg(pos + 4 * (long long)p0 + 3), d1 = __ldg(pos + 4 * (long long)p1 + 3);
            T d2 = __ldg(pos + 4 * (long long)p2 + 3), d3 = __ldg(pos + 4 * (long long)p3 + 3);
            cell_sum.add(pi_over_6<T>() * d0 * d0 * d0);
            cell_sum.add(pi_over_6<T>() * d1 * d1 * d1);
            cell_sum.add(pi_over_6<T>() * d2 * d2 * d2);
            cell_sum.add(pi_over_6<T>() * d3 * d3 * d3);
        }
        for (; i < e; ++i) {
            T d = __ldg(pos + 4 * (long long)__ldg(perm + i) + 3);
            cell_sum.add(pi_over_6<T>() * d * d * d);
        }
        const double vol = (double)cell_sum.s + (double)cell_sum.c;
        eps[c] = 1.0 - vol * g.invVB;
    }
    if (do_sums) {
        CSum<T> v[1] = {cell_sum};
        block_sums<T, 1>(v, part, pstride);
    }
}

// ----------------------------------------------------------------------
// Reaction source from the drag forces
//   SORTED: forces already in bin order as T4 (the fused drag output)
//   else  : caller-order SoA forces gathered through perm
// ----------------------------------------------------------------------
template <typename T, bool SORTED>
__global__ void __launch_bounds__(256)
k_deposit_momentum(const T* __restrict__ Fs, const T* __restrict__ F, long long n,
                   const int32_t* __restrict__ perm, const int32_t* __restrict__ cs, GridDev g,
                   T* __restrict__ S, double* __restrict__ part, long long pstride, int do_sums) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    CSum<T> a[3];
    CSum<T> sv[3];
    if (c < g.nbulk) {
        const int b = __ldg(cs + c), e = __ldg(cs + c + 1);
        for (int i = b; i < e; ++i) {
            if (SORTED) {
                V4<T> f = ld4(Fs, i);
                a[0].add(f.x);
                a[1].add(f.y);
                a[2].add(f.z);
            } else {
                const long long p = __ldg(perm + i);
                a[0].add(__ldg(F + p));
                a[1].add(__ldg(F + n + p));
                a[2].add(__ldg(F + 2 * n + p));
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T s;
            if (sizeof(T) == 4) s = -(a[k].get()) * (T)g.invVBf;
            else s = -(a[k].get()) * (T)g.invVB;
            S[k * g.nbulk + c] = s;
            // S_B V_B as an exact float-float product, V_B split in two
            if (sizeof(T) == 4) {
                T hi = s * (T)g.VBh;
                T lo = fma(s, (T)g.VBh, -hi);
                lo = fma(s, (T)g.VBl, lo);
                sv[k].add(hi);
                sv[k].c += lo;
            } else {
                sv[k].add(s * (T)g.VB);
            }
        }
    }
    if (do_sums) block_sums<T, 3>(sv, part, pstride);
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
    long long off[CG_NSUMS];     // offset of the partial column, -1 = not computed
    long long cnt[CG_NSUMS];     // number of partials
};

__global__ void __launch_bounds__(256) k_sums(const double* __restrict__ part, SumsMap map,
                                              double* __restrict__ sums) {
    __shared__ double sh_s[8], sh_c[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < CG_NSUMS; ++k) {
        CSum<double> a;
        if (map.off[k] >= 0)
            for (long long i = threadIdx.x; i < map.cnt[k]; i += blockDim.x) a.add(part[map.off[k] + i]);
        a = warp_reduce(a);
        if (lane == 0) {
            sh_s[warp] = a.s;
            sh_c[warp] = a.c;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            CSum<double> t;
            t.s = sh_s[0];
            t.c = sh_c[0];
            for (int w = 1; w < 8; ++w) {
                CSum<double> o;
                o.s = sh_s[w];
                o.c = sh_c[w];
                t.merge(o);
            }
            sums[k] = map.off[k] >= 0 ? t.get() : __longlong_as_double(0x7ff8000000000000LL);
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------
// Launchers
// ----------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int per) { return (unsigned)((n + per - 1) / per); }

cg_status launch_deposit_volume(cg_grids* g, long long n, const void* pos_d, double* eps, bool sums) {
    (void)n;
    const unsigned nblk = blocks_for(g->gd.nbulk, 256);
    double* part = g->partials + g->part_off[PS_VOL];
    g->part_blocks[PS_VOL] = sums ? (long long)nblk : -1;
    if (g->fp64)
        CG_LAUNCH(g, "deposit_volume", k_deposit_volume<double>, nblk, 256, 0, (const double*)pos_d, g->perm,
                  g->cell_start, g->gd, eps, part, (long long)nblk, (int)sums);
    else
        CG_LAUNCH(g, "deposit_volume", k_deposit_volume<float>, nblk, 256, 0, (const float*)pos_d, g->perm,
                  g->cell_start, g->gd, eps, part, (long long)nblk, (int)sums);
    return CG_OK;
}

cg_status launch_deposit_momentum(cg_grids* g, long long n, const void* force_soa, bool sorted, void* S_bulk,
                                  bool sums) {
    const unsigned nblk = blocks_for(g->gd.nbulk, 256);
    double* part = g->partials + g->part_off[PS_MOM];
    g->part_blocks[PS_MOM] = sums ? (long long)nblk : -1;
    if (g->fp64) {
        if (sorted)
            CG_LAUNCH(g, "deposit_momentum", (k_deposit_momentum<double, true>), nblk, 256, 0,
                      (const double*)g->Fs, nullptr, n, g->perm, g->cell_start, g->gd, (double*)S_bulk, part,
                      (long long)nblk, (int)sums);
        else
            CG_LAUNCH(g, "deposit_momentum", (k_deposit_momentum<double, false>), nblk, 256, 0, nullptr,
                      (const double*)force_soa, n, g->perm, g->cell_start, g->gd, (double*)S_bulk, part,
                      (long long)nblk, (int)sums);
    } else {
        if (sorted)
            CG_LAUNCH(g, "deposit_momentum", (k_deposit_momentum<float, true>), nblk, 256, 0,
                      (const float*)g->Fs, nullptr, n, g->perm, g->cell_start, g->gd, (float*)S_bulk, part,
                      (long long)nblk, (int)sums);
        else
            CG_LAUNCH(g, "deposit_momentum", (k_deposit_momentum<float, false>), nblk, 256, 0, nullptr,
                      (const float*)force_soa, n, g->perm, g->cell_start, g->gd, (float*)S_bulk, part,
                      (long long)nblk, (int)sums);
    }
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
        col(5 + a, PS_MOM, a);
        col(8 + a, PS_PROJ, a);
        col(12 + a, PS_DRAG, 5 + a);
    }
    col(11, PS_DRAG, 4);
    col(15, PS_DRAG, 8);
    CG_LAUNCH(g, "sums", k_sums, 1, 256, 0, g->partials, m, sums);
    return CG_OK;
}

}  // namespace cg
