// fine.cu -- the two fine-grid sweeps of the coupling step (Fig. 1 of
// arXiv 1807.11834): (a2) the fluid solution goes fine -> bulk, (a4) the
// particle-related fields go bulk -> fine.
//
// Both kernels run one thread per bulk cell.  Thread (I, J, K) owns the
// r^3 nested fine cells of its bulk cell: it reads (or writes) r^2 rows of
// r consecutive fine values per component, as one 16-byte vector per row
// for r = 4 (8 bytes for r = 2, two 16-byte vectors for r = 8).  Adjacent
// threads own adjacent bulk cells along x, so a warp touches 32 * r
// consecutive fine values per row: fully coalesced, every fine value read
// or written exactly once.  These two sweeps carry most of the bytes of a
// step, so they are written to stream at HBM speed.
#include <algorithm>

#include "cg_internal.cuh"
#include "batch.cuh"

namespace cg {

template <typename T, int R> struct Row;
template <> struct Row<float, 4> {
    static __device__ __forceinline__ void load(const float* p, float v[4]) {
        float4 q = __ldcs(reinterpret_cast<const float4*>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    static __device__ __forceinline__ void store(float* p, const float v[4]) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
    }
};
template <> struct Row<float, 2> {
    static __device__ __forceinline__ void load(const float* p, float v[2]) {
        float2 q = __ldcs(reinterpret_cast<const float2*>(p));
        v[0] = q.x; v[1] = q.y;
    }
    static __device__ __forceinline__ void store(float* p, const float v[2]) {
        __stcs(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
    }
};
template <> struct Row<float, 8> {
    static __device__ __forceinline__ void load(const float* p, float v[8]) {
        float4 a = __ldcs(reinterpret_cast<const float4*>(p)), b = __ldcs(reinterpret_cast<const float4*>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
    static __device__ __forceinline__ void store(float* p, const float v[8]) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
        __stcs(reinterpret_cast<float4*>(p) + 1, make_float4(v[4], v[5], v[6], v[7]));
    }
};
template <int R> struct Row<double, R> {
    static __device__ __forceinline__ void load(const double* p, double v[R]) {
#pragma unroll
        for (int i = 0; i < R; i += 2) {
            double2 q = __ldcs(reinterpret_cast<const double2*>(p + i));
            v[i] = q.x;
            v[i + 1] = q.y;
        }
    }
    static __device__ __forceinline__ void store(double* p, const double v[R]) {
#pragma unroll
        for (int i = 0; i < R; i += 2) __stcs(reinterpret_cast<double2*>(p + i), make_double2(v[i], v[i + 1]));
    }
};

__device__ __forceinline__ void bulk_ijk(long long cb, const GridDev& g, int& I, int& J, int& K) {
    I = (int)(cb % g.nb[0]);
    long long t = cb / g.nb[0];
    J = (int)(t % g.nb[1]);
    K = (int)(t / g.nb[1]);
}

// ----------------------------------------------------------------------
// (a2) mean and variance of the r^3 fine cells of a bulk cell, r = 2, 4, 8.
// The values are first shifted by the cell's first value (the subtraction
// is exact for values within a factor two of it), so that nothing below
// carries the mean's magnitude.  Pairwise over the rows of r values: each
// row gives its sum S and squared deviations M = sum (d - S/r)^2, and two
// sets of k values each merge as (S_a + S_b, M_a + M_b + (S_b - S_a)^2 / (2k))
// (the pairwise update of Chan, Golub & LeVeque), in a fixed binary tree
// over the r^2 rows; every division is by a power of two.
// ----------------------------------------------------------------------
template <typename T, int RC>
__device__ __forceinline__ void average_cell_pairwise(const T* __restrict__ u, const GridDev& g, T* __restrict__ ub,
                                                      T* __restrict__ var, long long cb, T* __restrict__ rec) {
    constexpr int NR = RC * RC;                                  // rows of a bulk cell
    constexpr int LV = RC == 2 ? 2 : RC == 4 ? 4 : 6;            // log2(NR)
    int I, J, K;
    bulk_ijk(cb, g, I, J, K);
    const long long nx = g.nf[0], nxy = (long long)g.nf[0] * g.nf[1];
    const long long f0 = (long long)I * RC + nx * ((long long)J * RC) + nxy * ((long long)K * RC);
    T stS[3][LV + 1], stM[3][LV + 1], ref[3];
    // rows are loaded AHEAD at a time (all their loads in flight together),
    // then merged one by one in the same order
    constexpr int AHEAD = (sizeof(T) == 4 && RC <= 4) ? (NR < 8 ? NR : 8) : (NR < 4 ? NR : 4);
#pragma unroll
    for (int r0 = 0; r0 < NR; r0 += AHEAD) {
    T vr[AHEAD][3][RC];
#pragma unroll
    for (int rr = 0; rr < AHEAD; ++rr) {
        const int r = r0 + rr;
        const long long f = f0 + nx * (r % RC) + nxy * (r / RC);
#pragma unroll
        for (int c = 0; c < 3; ++c) Row<T, RC>::load(u + c * g.nfine + f, vr[rr][c]);
    }
#pragma unroll
    for (int rr = 0; rr < AHEAD; ++rr) {
        const int r = r0 + rr;
        T (&v)[3][RC] = vr[rr];
        if (r == 0)
#pragma unroll
            for (int c = 0; c < 3; ++c) ref[c] = v[c][0];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int i = 0; i < RC; ++i) v[c][i] -= ref[c];
            // the row: pairwise sum, then squared deviations from its mean
            T w[RC];
#pragma unroll
            for (int i = 0; i < RC; ++i) w[i] = v[c][i];
#pragma unroll
            for (int h = RC / 2; h >= 1; h /= 2)
#pragma unroll
                for (int i = 0; i < h; ++i) w[i] = w[2 * i] + w[2 * i + 1];
            T S = w[0];
            const T mean = S * (T(1) / T(RC));
            T M = T(0);
#pragma unroll
            for (int i = 0; i < RC; ++i) {
                const T d = v[c][i] - mean;
                M = fma(d, d, M);
            }
            // merge up the tree while the row index has trailing ones
            T k = T(RC);
#pragma unroll
            for (int L = 0; L < LV; ++L) {
                if (((r >> L) & 1) == 0) {
                    stS[c][L] = S;
                    stM[c][L] = M;
                    break;
                }
                const T d = S - stS[c][L];
                M = stM[c][L] + M + d * d * (T(0.5) / k);
                S = stS[c][L] + S;
                k *= T(2);
                if (L == LV - 1) {
                    stS[c][LV] = S;
                    stM[c][LV] = M;
                }
            }
        }
    }
    }
    constexpr T invn = T(1) / T(RC * RC * RC);
    T m2 = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T mean = ref[c] + stS[c][LV] * invn;
        ub[c * g.nbulk + cb] = mean;
        if (rec) rec[4 * cb + 1 + c] = mean;
        m2 += stM[c][LV];
    }
    if (var) var[cb] = m2 * invn;
}

// ----------------------------------------------------------------------
// (a2) mean and variance of the r^3 fine cells of a bulk cell, any r.
// The variance uses a shift by the first fine value of the cell:
// var = (Q - sum_c D_c^2 / n) / n with Q = sum (u - ref)^2 and
// D_c = sum_f u_c - n ref_c, both compensated, which equals the two-pass
// population variance without a second read of the fine data.
// ----------------------------------------------------------------------
// rec (nullable): the drag's packed record (eps, u_x, u_y, u_z) per cell;
// the mean velocity is also written to its u part.
template <typename T, int RC>
__device__ __forceinline__ void average_cell(const T* __restrict__ u, const GridDev& g, T* __restrict__ ub,
                                             T* __restrict__ var, long long cb, T* __restrict__ rec);

template <typename T, int RC>
__device__ __forceinline__ void average_body(const T* __restrict__ u, const GridDev& g, T* __restrict__ ub,
                                             T* __restrict__ var, Blk b, T* __restrict__ rec = nullptr) {
    for (long long cb = b.id * blockDim.x + threadIdx.x; cb < g.nbulk; cb += b.n * blockDim.x) {
        if constexpr (RC > 0) average_cell_pairwise<T, RC>(u, g, ub, var, cb, rec);
        else average_cell<T, RC>(u, g, ub, var, cb, rec);
    }
}

template <typename T, int RC>
__global__ void __launch_bounds__(256, 2)
k_average(const T* __restrict__ u, GridDev g, T* __restrict__ ub, T* __restrict__ var, T* __restrict__ rec) {
    pdl_wait();
    average_body<T, RC>(u, g, ub, var, launch_blk(), rec);
}

template <typename T, int RC>
__device__ __forceinline__ void average_cell(const T* __restrict__ u, const GridDev& g, T* __restrict__ ub,
                                             T* __restrict__ var, long long cb, T* __restrict__ rec) {
    int I, J, K;
    bulk_ijk(cb, g, I, J, K);
    const int r = RC ? RC : g.r;
    const long long nx = g.nf[0], nxy = (long long)g.nf[0] * g.nf[1];
    const long long f0 = (long long)I * r + nx * ((long long)J * r) + nxy * ((long long)K * r);
    CSum<T> s[3], q;
    T ref[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) ref[c] = __ldg(u + c * g.nfine + f0);
    if constexpr (RC > 0) {
#pragma unroll
        for (int dk = 0; dk < RC; ++dk) {
#pragma unroll
            for (int dj = 0; dj < RC; ++dj) {
                const long long f = f0 + nx * dj + nxy * dk;
                T v[3][RC];
#pragma unroll
                for (int c = 0; c < 3; ++c) Row<T, RC>::load(u + c * g.nfine + f, v[c]);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int i = 0; i < RC; ++i) {
                        s[c].add(v[c][i]);
                        T dv = v[c][i] - ref[c];
                        q.add(dv * dv);
                    }
            }
        }
    } else {
        for (int dk = 0; dk < r; ++dk)
            for (int dj = 0; dj < r; ++dj) {
                const long long f = f0 + nx * dj + nxy * dk;
                for (int i = 0; i < r; ++i)
                    for (int c = 0; c < 3; ++c) {
                        T v = __ldg(u + c * g.nfine + f + i);
                        s[c].add(v);
                        T dv = v - ref[c];
                        q.add(dv * dv);
                    }
            }
    }
    const T n = (T)r * (T)r * (T)r;
    const T invn = (T)1 / n;
    T corr = 0;
    T mean[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        mean[c] = s[c].get() * invn;
        ub[c * g.nbulk + cb] = mean[c];
        if (var) {
            // D_c = (s_hi - n ref) + s_lo, the n ref product split exactly
            T p = n * ref[c];
            T pe = fma(n, ref[c], -p);
            T d1, e1;
            two_sum(s[c].s, -p, d1, e1);
            T D = d1 + (e1 + (s[c].c - pe));
            corr += D * D;
        }
    }
    if (var) {
        T a, e;
        two_sum(q.s, -corr * invn, a, e);
        T v = (a + (e + q.c)) * invn;
        var[cb] = v > T(0) ? v : T(0);
    }
    if (rec)
#pragma unroll
        for (int c = 0; c < 3; ++c) rec[4 * cb + 1 + c] = mean[c];
}

// ----------------------------------------------------------------------
// (a4) interpolate ncomp bulk fields at the fine cell centres of a bulk
// cell.  Along one axis, fine offset a in [0, r) of bulk cell I sits at
// lattice coordinate xi = I + (2a + 1 - r) / (2r): for 2a + 1 < r it lies
// between bulk centres I-1 and I with t = (2a + 1 + r) / (2r), otherwise
// between I and I+1 with t = (2a + 1 - r) / (2r).  At the domain edges the
// neighbour index is clamped to I, which reproduces constant extrapolation
// in the outer half cell exactly because lerp(a, a, t) == a.  The weights
// are exact dyadic rationals for power-of-two r.
// ----------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T lerp(T a, T b, T t) { return fma(t, b - a, a); }

template <int R> struct Stencil {
    // neighbour slot (0: I-1, 1: I, 2: I+1) of the lower/upper support and t
    static __device__ __forceinline__ void at(int a, int& lo, int& hi, float& t) {
        const int num = 2 * a + 1 - R;
        if (num < 0) { lo = 0; hi = 1; t = (float)(num + 2 * R) / (float)(2 * R); }
        else { lo = 1; hi = 2; t = (float)num / (float)(2 * R); }
    }
};

// Multiply a compensated sum by V_f, keeping the product's rounding error.
__device__ __forceinline__ void scale_sum(CSum<float>& a, const GridDev& g) {
    float hi = a.s * g.Vfh;
    float lo = fmaf(a.s, g.Vfh, -hi);
    lo = fmaf(a.s, g.Vfl, lo);
    lo = fmaf(a.c, g.Vfh, lo);
    a.s = hi;
    a.c = lo;
}
__device__ __forceinline__ void scale_sum(CSum<double>& a, const GridDev& g) {
    a.s *= g.Vf;
    a.c *= g.Vf;
}

// S_B V_B of one bulk cell into a conservation sum: an exact float-float
// product on the FP32 path (the reaction deposit's S_B = -(1/V_B) sum F,
// so the sums of S_B V_B and of the forces cancel to the compensated sums'
// accuracy).
__device__ __forceinline__ void add_bulk_term(CSum<float>& a, float sb, const GridDev& g) {
    const float hi = sb * g.VBh;
    float lo = fmaf(sb, g.VBh, -hi);
    lo = fmaf(sb, g.VBl, lo);
    a.add(hi);
    a.c += lo;
}
__device__ __forceinline__ void add_bulk_term(CSum<double>& a, double sb, const GridDev& g) { a.add(sb * g.VB); }

// One thread per bulk cell (block b covers cells [b.id blockDim, (b.id + 1) blockDim)).
template <typename T, int RC>
__device__ __forceinline__ void project_body(const T* __restrict__ in0, const T* __restrict__ in1,
                                             const T* __restrict__ in2, const T* __restrict__ in3, int ncomp,
                                             const GridDev& g, T* __restrict__ out0, T* __restrict__ out1,
                                             T* __restrict__ out2, T* __restrict__ out3, T* __restrict__ part,
                                             long long pstride, int do_sums, Blk b) {
    const long long cb = b.id * blockDim.x + threadIdx.x;
    CSum<T> sacc[6];   // sum_f S_f (3), then sum S_B V_B of this thread's bulk cell (3)
    if (cb < g.nbulk) {
        int I, J, K;
        bulk_ijk(cb, g, I, J, K);
        const int nbx = g.nb[0], nby = g.nb[1], nbz = g.nb[2];
        const int xs[3] = {max(I - 1, 0), I, min(I + 1, nbx - 1)};
        const int ys[3] = {max(J - 1, 0), J, min(J + 1, nby - 1)};
        const int zs[3] = {max(K - 1, 0), K, min(K + 1, nbz - 1)};
        const long long nx = g.nf[0], nxy = (long long)g.nf[0] * g.nf[1];
        const long long f0 = (long long)I * RC + nx * ((long long)J * RC) + nxy * ((long long)K * RC);
#pragma unroll 1
        for (int c = 0; c < ncomp; ++c) {
            const T* __restrict__ B = c == 0 ? in0 : c == 1 ? in1 : c == 2 ? in2 : in3;
            T* __restrict__ O = c == 0 ? out0 : c == 1 ? out1 : c == 2 ? out2 : out3;
            T f[3][3][3];   // [z][y][x]
            if (g.interp == CG_INTERP_CELL) {
                // cell values: every nested fine cell takes its bulk cell's value
                const T v0 = __ldg(B + cb);
#pragma unroll
                for (int z = 0; z < 3; ++z)
#pragma unroll
                    for (int y = 0; y < 3; ++y)
#pragma unroll
                        for (int x = 0; x < 3; ++x) f[z][y][x] = v0;
            } else {
#pragma unroll
                for (int z = 0; z < 3; ++z)
#pragma unroll
                    for (int y = 0; y < 3; ++y)
#pragma unroll
                        for (int x = 0; x < 3; ++x)
                            f[z][y][x] = __ldg(B + xs[x] + (long long)nbx * (ys[y] + (long long)nby * zs[z]));
            }
            CSum<T> rowsum;
#pragma unroll
            for (int az = 0; az < RC; ++az) {
                int zlo, zhi;
                float tzf;
                Stencil<RC>::at(az, zlo, zhi, tzf);
                const T tz = (T)tzf;
                T fz[3][3];   // [y][x] after the z lerp
#pragma unroll
                for (int y = 0; y < 3; ++y)
#pragma unroll
                    for (int x = 0; x < 3; ++x) fz[y][x] = lerp(f[zlo][y][x], f[zhi][y][x], tz);
#pragma unroll
                for (int ay = 0; ay < RC; ++ay) {
                    int ylo, yhi;
                    float tyf;
                    Stencil<RC>::at(ay, ylo, yhi, tyf);
                    const T ty = (T)tyf;
                    T gx[3];
#pragma unroll
                    for (int x = 0; x < 3; ++x) gx[x] = lerp(fz[ylo][x], fz[yhi][x], ty);
                    T v[RC];
                    T rs = 0;
#pragma unroll
                    for (int ax = 0; ax < RC; ++ax) {
                        int xlo, xhi;
                        float txf;
                        Stencil<RC>::at(ax, xlo, xhi, txf);
                        v[ax] = lerp(gx[xlo], gx[xhi], (T)txf);
                        rs += v[ax];
                    }
                    Row<T, RC>::store(O + f0 + nx * ay + nxy * az, v);
                    rowsum.add(rs);
                }
            }
            if (c < 3) {
                sacc[c] = rowsum;
                add_bulk_term(sacc[3 + c], f[1][1][1], g);   // the stencil's centre: this cell's S_B
            }
        }
    }
    if (do_sums) {
        // sum_f S_f V_f = V_f sum_f S_f; V_f applied as a float-float product
#pragma unroll
        for (int c = 0; c < 3; ++c) scale_sum(sacc[c], g);
        block_sums<T, 6>(sacc, part, pstride, b.id);
    }
}

template <typename T, int RC>
__global__ void __launch_bounds__(256)
k_project(const T* __restrict__ in0, const T* __restrict__ in1, const T* __restrict__ in2,
          const T* __restrict__ in3, int ncomp, GridDev g, T* __restrict__ out0, T* __restrict__ out1,
          T* __restrict__ out2, T* __restrict__ out3, T* __restrict__ part, long long pstride,
          int do_sums) {
    pdl_wait();
    project_body<T, RC>(in0, in1, in2, in3, ncomp, g, out0, out1, out2, out3, part, pstride, do_sums,
                        launch_blk());
}

// Generic ratio: one thread per fine cell, the same clamped stencil with
// integer-derived weights.
template <typename T>
__global__ void __launch_bounds__(256)
k_project_generic(const T* __restrict__ in0, const T* __restrict__ in1, const T* __restrict__ in2,
                  const T* __restrict__ in3, int ncomp, GridDev g, T* __restrict__ out0,
                  T* __restrict__ out1, T* __restrict__ out2, T* __restrict__ out3,
                  T* __restrict__ part, long long pstride, int do_sums) {
    pdl_wait();
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    CSum<T> sacc[6];   // sum_f S_f (3), then sum S_B V_B (3, from each bulk cell's lower-corner fine cell)
    if (f < g.nfine) {
        const int r = g.r;
        long long t = f;
        const int fi[3] = {(int)(t % g.nf[0]), (int)((t / g.nf[0]) % g.nf[1]),
                           (int)(t / ((long long)g.nf[0] * g.nf[1]))};
        int lo[3], hi[3];
        T w[3];
        for (int a = 0; a < 3; ++a) {
            const int I = fi[a] / r, off = fi[a] - I * r;
            const int num = 2 * off + 1 - r;
            if (g.interp == CG_INTERP_CELL) { lo[a] = hi[a] = I; w[a] = T(0); }
            else if (num < 0) { lo[a] = max(I - 1, 0); hi[a] = I; w[a] = (T)(num + 2 * r) / (T)(2 * r); }
            else { lo[a] = I; hi[a] = min(I + 1, g.nb[a] - 1); w[a] = (T)num / (T)(2 * r); }
        }
        const long long nbx = g.nb[0], nbxy = (long long)g.nb[0] * g.nb[1];
        for (int c = 0; c < ncomp; ++c) {
            const T* __restrict__ B = c == 0 ? in0 : c == 1 ? in1 : c == 2 ? in2 : in3;
            T* __restrict__ O = c == 0 ? out0 : c == 1 ? out1 : c == 2 ? out2 : out3;
            T zv[2];
            for (int dz = 0; dz < 2; ++dz) {
                const long long kz = (dz ? hi[2] : lo[2]) * nbxy;
                T yv[2];
                for (int dy = 0; dy < 2; ++dy) {
                    const long long jy = (dy ? hi[1] : lo[1]) * nbx;
                    yv[dy] = lerp(__ldg(B + kz + jy + lo[0]), __ldg(B + kz + jy + hi[0]), w[0]);
                }
                zv[dz] = lerp(yv[0], yv[1], w[1]);
            }
            const T v = lerp(zv[0], zv[1], w[2]);
            O[f] = v;
            if (c < 3) {
                sacc[c].add(v);
                if (fi[0] % r == 0 && fi[1] % r == 0 && fi[2] % r == 0)
                    add_bulk_term(sacc[3 + c], __ldg(B + (fi[2] / r) * nbxy + (fi[1] / r) * nbx + fi[0] / r), g);
            }
        }
    }
    if (do_sums) {
#pragma unroll
        for (int c = 0; c < 3; ++c) scale_sum(sacc[c], g);
        block_sums<T, 6>(sacc, part, pstride, blockIdx.x);
    }
}

// ----------------------------------------------------------------------
// Batched fine-grid phases (FP32 instances, ratio 2, 4 or 8)
// ----------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) kb_average(BLaunch L) {
    batch_loop(L, [&](const BInst& I, Blk b) {
        switch (I.gd.r) {
            case 2: average_body<float, 2>(I.u_fine, I.gd, I.u_bulk, I.var, b); break;
            case 4: average_body<float, 4>(I.u_fine, I.gd, I.u_bulk, I.var, b); break;
            default: average_body<float, 8>(I.u_fine, I.gd, I.u_bulk, I.var, b); break;
        }
    });
}

// eps: project the porosity (one component, no sums) instead of the source
__global__ void __launch_bounds__(256) kb_project(BLaunch L, int eps) {
    batch_loop(L, [&](const BInst& I, Blk b) {
        const long long nb = I.gd.nbulk, nf = I.gd.nfine;
        const float* in0 = eps ? I.eps_t : I.S_bulk;
        const float* in1 = eps ? nullptr : I.S_bulk + nb;
        const float* in2 = eps ? nullptr : I.S_bulk + 2 * nb;
        float* o0 = eps ? I.eps_fine : I.S_fine;
        float* o1 = eps ? nullptr : I.S_fine + nf;
        float* o2 = eps ? nullptr : I.S_fine + 2 * nf;
        const int nc = eps ? 1 : 3;
        float* part = I.part + 2 * I.part_off[PS_PROJ];
        const long long ps = I.part_blocks[PS_PROJ];
        switch (I.gd.r) {
            case 2: project_body<float, 2>(in0, in1, in2, nullptr, nc, I.gd, o0, o1, o2, nullptr, part, ps, !eps, b); break;
            case 4: project_body<float, 4>(in0, in1, in2, nullptr, nc, I.gd, o0, o1, o2, nullptr, part, ps, !eps, b); break;
            default: project_body<float, 8>(in0, in1, in2, nullptr, nc, I.gd, o0, o1, o2, nullptr, part, ps, !eps, b); break;
        }
    });
}

cg_status launch_batch_fine(int phase, const BLaunch& L, unsigned grid, cudaStream_t s) {
    if (L.total == 0 || grid == 0) return CG_OK;
    switch (phase) {
        case BP_AVG: kb_average<<<grid, 256, 0, s>>>(L); break;
        case BP_PROJ: kb_project<<<grid, 256, 0, s>>>(L, 0); break;
        case BP_PROJE: kb_project<<<grid, 256, 0, s>>>(L, 1); break;
        default: return CG_ERR_INVALID_ARG;
    }
    CG_CUDA(cudaGetLastError());
    return CG_OK;
}

int batch_fine_occupancy(int phase) {
    int occ = 0;
    cudaError_t e = phase == BP_AVG ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_average, 256, 0)
                                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_project, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return occ > 0 ? occ : 1;
}

static inline unsigned blocks_of(long long n, int per) { return (unsigned)((n + per - 1) / per); }

cg_status launch_average(cg_grids* g, const void* u_fine, void* u_bulk, void* var_bulk, void* rec) {
    // grid-stride over one block per SM: each thread keeps 8 rows x 3
    // components of loads in flight (about 100 registers), enough to stream
    // near HBM speed while leaving most warp slots and registers to the
    // particle kernels running beside it (two blocks per SM ran the average
    // alone as fast but slowed the step by 12 us)
    const unsigned nblk = (unsigned)std::min((long long)blocks_of(g->gd.nbulk, 256), (long long)g->num_sms * 1);
#define CG_AVG(T, RC)                                                                                   \
    CG_LAUNCH(g, "average", (k_average<T, RC>), nblk, 256, 0, (const T*)u_fine, g->gd, (T*)u_bulk, \
              (T*)var_bulk, (T*)rec)
    if (g->fp64) {
        switch (g->gd.r) {
            case 2: CG_AVG(double, 2); break;
            case 4: CG_AVG(double, 4); break;
            case 8: CG_AVG(double, 8); break;
            default: CG_AVG(double, 0); break;
        }
    } else {
        switch (g->gd.r) {
            case 2: CG_AVG(float, 2); break;
            case 4: CG_AVG(float, 4); break;
            case 8: CG_AVG(float, 8); break;
            default: CG_AVG(float, 0); break;
        }
    }
#undef CG_AVG
    return CG_OK;
}

cg_status launch_project(cg_grids* g, int ncomp, const void* const* in, void* const* out, bool sums) {
    void* part = part_ptr(g, PS_PROJ);
    const int r = g->gd.r;
    const bool fast = (r == 2 || r == 4 || r == 8);
    const unsigned nblk = fast ? blocks_of(g->gd.nbulk, 256) : blocks_of(g->gd.nfine, 256);
    // only the projection that forms the sums claims their partials (a later
    // projection without sums, of the porosity or the semi-implicit
    // coefficients, leaves them to it)
    if (sums) g->part_blocks[PS_PROJ] = (long long)nblk;
#define CG_PRJ(T, KER)                                                                                   \
    CG_LAUNCH(g, ncomp == 1 ? "project_eps" : ncomp == 4 ? "project_implicit" : "project", KER, nblk, 256, 0, (const T*)in[0], (const T*)in[1], (const T*)in[2], \
              (const T*)in[3], ncomp, g->gd, (T*)out[0], (T*)out[1], (T*)out[2], (T*)out[3], (T*)part,   \
              (long long)nblk, (int)sums)
    if (g->fp64) {
        switch (r) {
            case 2: CG_PRJ(double, (k_project<double, 2>)); break;
            case 4: CG_PRJ(double, (k_project<double, 4>)); break;
            case 8: CG_PRJ(double, (k_project<double, 8>)); break;
            default: CG_PRJ(double, k_project_generic<double>); break;
        }
    } else {
        switch (r) {
            case 2: CG_PRJ(float, (k_project<float, 2>)); break;
            case 4: CG_PRJ(float, (k_project<float, 4>)); break;
            case 8: CG_PRJ(float, (k_project<float, 8>)); break;
            default: CG_PRJ(float, k_project_generic<float>); break;
        }
    }
#undef CG_PRJ
    return CG_OK;
}

}  // namespace cg
