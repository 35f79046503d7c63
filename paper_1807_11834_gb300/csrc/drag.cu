// drag.cu -- (a3) drag on every particle, Eq. (DragLaw) of arXiv 1807.11834:
// F = beta (u_f - u_p), with the porosity and the fluid velocity taken at the
// particle from the bulk grid (the cell value or a local interpolant,
// Sec. 1), and beta from a correlation of slip, densities, diameter,
// viscosity and porosity.  Optionally (a5) the semi-implicit Euler advance
// of Eq. (DEM_EQUATIONS) without contacts.
//
// One thread per particle in the caller's order: the particle record is
// read once (two 16-byte loads) and the force written once (three
// coalesced stores).  The bulk fields are gathered from a packed array of
// (eps, u_x, u_y, u_z) per cell, eight 16-byte loads that stay in L2.  For
// the fused reaction deposit the force is also written, as a 16-byte
// record, to its slot in bin order, so the following segmented sum reads
// it contiguously.
//
// FP32 path: the lattice coordinate (x - x0)/H - 1/2 is formed in
// float-float (FMA TwoProduct and one TwoSum), so the interpolation weights
// carry only the final float rounding even at |xi| ~ 100; the correlations
// run in float with explicitly rounded operations, their powers, logarithm,
// roots and reciprocals on the special-function unit (drag_law.cuh).
// On request (CG_STENCIL_WINDOW) the sorted step stages each warp's stencil
// window in shared memory instead of gathering from L2 (window_gather).
#include <algorithm>

#include "cg_internal.cuh"
#include "drag_law.cuh"
#include "batch.cuh"

namespace cg {

template <typename T>
__device__ __forceinline__ V4<T> ld4_plain(const T* p, long long i) {
    if (sizeof(T) == 4) {
        float4 v = reinterpret_cast<const float4*>(p)[i];
        return {(T)v.x, (T)v.y, (T)v.z, (T)v.w};
    } else {
        const double2* q = reinterpret_cast<const double2*>(p) + 2 * i;
        double2 a = q[0], b = q[1];
        return {(T)a.x, (T)a.y, (T)b.x, (T)b.y};
    }
}

// ----------------------------------------------------------------------
// One particle: the porosity and fluid velocity gathered at x, the drag
// force, and with EULER the advanced state (else x and u unchanged).
// ----------------------------------------------------------------------
template <typename T>
struct DragOne {
    T f[3], beta, smag, vp, m, x[3], u[3];
    int cl;
};

template <typename T, bool EULER>
__device__ __forceinline__ DragOne<T> drag_from(const V4<T>& x, const V4<T>& v, const V4<T>& b, const GridDev& g,
                                                const Phys<T>& P, T dt) {
    using X = M<T>;
    DragOne<T> r;
    T eps = b.x;
    T phi = X::sub(T(1), eps);
    r.cl = 0;
    if (eps < P.eps_min) {
        eps = P.eps_min;
        phi = X::sub(T(1), P.eps_min);
        r.cl = 1;
    }
    const T sx = X::sub(b.y, v.x), sy = X::sub(b.z, v.y), sz = X::sub(b.w, v.z);
    r.smag = X::sqrt_(X::fma_(sx, sx, X::fma_(sy, sy, X::mul(sz, sz))));
    const T d = x.w;
    r.beta = drag_beta(g.law, eps, phi, d, r.smag, P);
    r.f[0] = X::mul(r.beta, sx);
    r.f[1] = X::mul(r.beta, sy);
    r.f[2] = X::mul(r.beta, sz);
    r.vp = X::mul(X::mul(X::mul(M<T>::pi6(), d), d), d);
    r.m = X::mul(P.rho_p, r.vp);
    r.x[0] = x.x;
    r.x[1] = x.y;
    r.x[2] = x.z;
    r.u[0] = v.x;
    r.u[1] = v.y;
    r.u[2] = v.z;
    if (EULER) {
        const T inv_m = X::rcp_(r.m);   // one reciprocal for the three components
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            T ua = X::fma_(dt, X::fma_(r.f[a], inv_m, P.g[a]), r.u[a]);
            T xa = X::fma_(dt, ua, r.x[a]);
            // the FP32 path reads the bounds' float copies (no conversion in the loop)
            const T lo = sizeof(T) == 4 ? (T)g.x0f[a] : (T)g.x0[a];
            const T hi = sizeof(T) == 4 ? (T)g.xhif[a] : (T)g.xhi[a];
            if (xa < lo) { xa = X::sub(X::mul(T(2), lo), xa); ua = -ua; }
            else if (xa > hi) { xa = X::sub(X::mul(T(2), hi), xa); ua = -ua; }
            r.x[a] = xa;
            r.u[a] = ua;
        }
    }
    return r;
}

template <typename T, bool EULER>
__device__ __forceinline__ DragOne<T> drag_one(const V4<T>& x, const V4<T>& v, const GridDev& g, const Phys<T>& P,
                                               const T* __restrict__ bulk4, T dt) {
    return drag_from<T, EULER>(x, v, gather(bulk4, x.x, x.y, x.z, g), g, P, dt);
}

// Stencil window of a warp (particles in cell order): the bounding box of
// the 32 particles' stencil base cells, grown by the +1 halo on each axis,
// staged from the bulk record into the warp's slice of shared memory with
// one 16-byte load per record (x rows contiguous), and each particle's
// eight corners read from there.  A box of more than kWinRecs records (the
// particles far apart: not in cell order) takes the gather from global
// memory.  Both give the same value (interp8).  All lanes of the warp call
// it together (valid: the lane holds a particle).
constexpr int kWinRecs = 64;
__device__ __forceinline__ void st_win(V4<float>* q, const V4<float>& v) {
    *reinterpret_cast<float4*>(q) = make_float4(v.x, v.y, v.z, v.w);
}
__device__ __forceinline__ void st_win(V4<double>* q, const V4<double>& v) {
    reinterpret_cast<double2*>(q)[0] = make_double2(v.x, v.y);
    reinterpret_cast<double2*>(q)[1] = make_double2(v.z, v.w);
}
__device__ __forceinline__ V4<float> ld_win(const V4<float>* q) {
    const float4 v = *reinterpret_cast<const float4*>(q);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ld_win(const V4<double>* q) {
    const double2 a = reinterpret_cast<const double2*>(q)[0], b = reinterpret_cast<const double2*>(q)[1];
    return {a.x, a.y, b.x, b.y};
}
template <typename T>
__device__ __forceinline__ V4<T> window_gather(const T* __restrict__ bulk4, const V4<T>& x, bool valid,
                                               const GridDev& g, V4<T>* __restrict__ win) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int i0 = 0, j0 = 0, k0 = 0;
    T tx = T(0), ty = T(0), tz = T(0);
    if (valid) {
        axis_weight(x.x, g, 0, i0, tx);
        axis_weight(x.y, g, 1, j0, ty);
        axis_weight(x.z, g, 2, k0, tz);
    }
    const int big = 0x7fffffff;
    const int imin = __reduce_min_sync(full, valid ? i0 : big), imax = __reduce_max_sync(full, valid ? i0 : -1);
    const int jmin = __reduce_min_sync(full, valid ? j0 : big), jmax = __reduce_max_sync(full, valid ? j0 : -1);
    const int kmin = __reduce_min_sync(full, valid ? k0 : big), kmax = __reduce_max_sync(full, valid ? k0 : -1);
    const int nx = imax - imin + 2, ny = jmax - jmin + 2, nz = kmax - kmin + 2;
    const int sy = g.nb[0], sz = g.nb[0] * g.nb[1];
    const V4<T>* rec = reinterpret_cast<const V4<T>*>(bulk4);
    V4<T> out = {T(0), T(0), T(0), T(0)};
    // the box is small only if every extent is (no product of large extents)
    if (nx <= kWinRecs && ny <= kWinRecs && nz <= kWinRecs && nx * ny * nz <= kWinRecs) {
        const int W = nx * ny * nz;
        // record r = wx + nx (wy + ny wz); (r + 1/2) / n never rounds across an integer for r < 2^11
        const float inx = 1.0f / (float)nx, iny = 1.0f / (float)ny;
        for (int r = lane; r < W; r += 32) {
            const int q = (int)(((float)r + 0.5f) * inx);
            const int wx = r - q * nx;
            const int wz = (int)(((float)q + 0.5f) * iny);
            const int wy = q - wz * ny;
            st_win(win + r, ldv4(rec + (imin + wx) + sy * (jmin + wy) + sz * (kmin + wz)));
        }
        __syncwarp();
        if (valid)
            out = interp8<T>(win + (i0 - imin) + nx * ((j0 - jmin) + ny * (k0 - kmin)), nx, nx * ny, tx, ty, tz,
                             [](const V4<T>* q) { return ld_win(q); });
        __syncwarp();   // the next call restages the slice
    } else if (valid) {
        out = interp8<T>(rec + (i0 + sy * j0 + sz * k0), sy, sz, tx, ty, tz, [](const V4<T>* q) { return ldv4(q); });
    }
    return out;
}

// Per-lane diagnostics: V_p, F (3), |F|, m u (3) after the advance, clamped.
template <typename T>
__device__ __forceinline__ void drag_lane_sums(T (&ls)[kDragSums], const DragOne<T>& r) {
    using X = M<T>;
    ls[0] = X::add(ls[0], r.vp);
    ls[1] = X::add(ls[1], r.f[0]);
    ls[2] = X::add(ls[2], r.f[1]);
    ls[3] = X::add(ls[3], r.f[2]);
    ls[4] = X::fma_(r.beta, r.smag, ls[4]);
    ls[5] = X::fma_(r.m, r.u[0], ls[5]);
    ls[6] = X::fma_(r.m, r.u[1], ls[6]);
    ls[7] = X::fma_(r.m, r.u[2], ls[7]);
    ls[8] = X::add(ls[8], (T)r.cl);
}

// ----------------------------------------------------------------------
// Drag kernel.  Partial sums (per block): V_p, F (3), |F|, m u (3), clamped.
// With EULER the particle is advanced in place after its force is known:
// u += dt (F/m + g), x += dt u, specular reflection at the domain faces.
// ----------------------------------------------------------------------
// Bs (nullable): the semi-implicit record (beta, beta u_p) of each particle,
// written to its sorted slot beside the force record.
// pos_out, vel_out (nullable, with Fs): the particle records, advanced when
// EULER, are written to their sorted slot of these arrays instead of in
// place (the sorted step: the particles leave in this binning's order).
template <typename T, bool EULER, bool PREFETCH = true>
__device__ __forceinline__ void drag_body(T* pos, T* vel, long long n, const GridDev& g, const Phys<T>& P,
                                          const T* __restrict__ bulk4, T* __restrict__ F, T* __restrict__ Fs,
                                          const int32_t* __restrict__ inv_perm, T dt, T* __restrict__ part,
                                          long long pstride, int do_sums, unsigned long long* __restrict__ status,
                                          Blk b, T* __restrict__ Bs = nullptr, T* __restrict__ pos_out = nullptr,
                                          T* __restrict__ vel_out = nullptr) {
    T lane_sums[kDragSums];
#pragma unroll
    for (int k = 0; k < kDragSums; ++k) lane_sums[k] = T(0);
    int clamped_total = 0;
    const long long stride = b.n * blockDim.x;
    // PREFETCH: the next particle's record is loaded while this one's
    // stencil is gathered and its force computed (its DRAM latency overlaps
    // them); the batched kernel, short of registers, loads it in turn
    V4<T> xn, vn;
    int slot_n = 0;
    long long p = b.id * blockDim.x + threadIdx.x;
    if (p < n) {
        xn = EULER ? ld4_plain(pos, p) : ld4((const T*)pos, p);
        vn = EULER ? ld4_plain(vel, p) : ld4((const T*)vel, p);
        if (Fs) slot_n = __ldg(inv_perm + p);
    }
    for (; p < n; p += stride) {
        if (!PREFETCH && p != b.id * blockDim.x + threadIdx.x) {
            xn = EULER ? ld4_plain(pos, p) : ld4((const T*)pos, p);
            vn = EULER ? ld4_plain(vel, p) : ld4((const T*)vel, p);
            if (Fs) slot_n = __ldg(inv_perm + p);
        }
        const V4<T> x = xn, v = vn;
        const int slot = slot_n;
        if (PREFETCH && p + stride < n) {
            xn = EULER ? ld4_plain(pos, p + stride) : ld4((const T*)pos, p + stride);
            vn = EULER ? ld4_plain(vel, p + stride) : ld4((const T*)vel, p + stride);
            if (Fs) slot_n = __ldg(inv_perm + p + stride);
        }
        const DragOne<T> r = drag_one<T, EULER>(x, v, g, P, bulk4, dt);
        clamped_total += r.cl;
        F[p] = r.f[0];
        F[n + p] = r.f[1];
        F[2 * n + p] = r.f[2];
        if (Fs) st4(Fs, slot, r.f[0], r.f[1], r.f[2], T(0));
        if (Bs) st4(Bs, slot, r.beta, r.beta * v.x, r.beta * v.y, r.beta * v.z);
        if (pos_out) {
            st4(pos_out, slot, r.x[0], r.x[1], r.x[2], x.w);
            st4(vel_out, slot, r.u[0], r.u[1], r.u[2], v.w);
        } else if (EULER) {
            st4(pos, p, r.x[0], r.x[1], r.x[2], x.w);
            st4(vel, p, r.u[0], r.u[1], r.u[2], v.w);
        }
        drag_lane_sums(lane_sums, r);
    }
    int wsum = clamped_total;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
    if ((threadIdx.x & 31) == 0 && wsum) {
        atomicAdd(&status[ST_CLAMPED], (unsigned long long)wsum);
        atomicOr(&status[ST_FLAGS], (unsigned long long)CG_FLAG_EPS_CLAMPED);
    }
    if (do_sums) {
        CSum<T> acc[kDragSums];
#pragma unroll
        for (int k = 0; k < kDragSums; ++k) acc[k].add(lane_sums[k]);
        block_sums<T, kDragSums>(acc, part, pstride, b.id);
    }
}

// The drag of particles in cell order (the sorted step) with the stencil
// window of each warp (window_gather); otherwise as drag_body, whose
// results it reproduces bit for bit.  The loop runs warp by warp (every
// lane of a warp takes the same number of turns).
template <typename T, bool EULER>
__device__ __forceinline__ void drag_body_win(T* pos, T* vel, long long n, const GridDev& g, const Phys<T>& P,
                                              const T* __restrict__ bulk4, T* __restrict__ F, T* __restrict__ Fs,
                                              const int32_t* __restrict__ inv_perm, T dt, T* __restrict__ part,
                                              long long pstride, int do_sums, unsigned long long* __restrict__ status,
                                              Blk b, T* __restrict__ pos_out, T* __restrict__ vel_out,
                                              V4<T>* __restrict__ win) {
    T lane_sums[kDragSums];
#pragma unroll
    for (int k = 0; k < kDragSums; ++k) lane_sums[k] = T(0);
    int clamped_total = 0;
    const long long stride = b.n * blockDim.x;
    const int lane = threadIdx.x & 31;
    V4<T> xn = {T(0), T(0), T(0), T(0)}, vn = xn;
    int slot_n = 0;
    long long p = b.id * blockDim.x + threadIdx.x;
    if (p < n) {
        xn = EULER ? ld4_plain(pos, p) : ld4((const T*)pos, p);
        vn = EULER ? ld4_plain(vel, p) : ld4((const T*)vel, p);
        slot_n = __ldg(inv_perm + p);
    }
    for (; p - lane < n; p += stride) {
        const bool valid = p < n;
        const V4<T> x = xn, v = vn;
        const int slot = slot_n;
        if (p + stride < n) {
            xn = EULER ? ld4_plain(pos, p + stride) : ld4((const T*)pos, p + stride);
            vn = EULER ? ld4_plain(vel, p + stride) : ld4((const T*)vel, p + stride);
            slot_n = __ldg(inv_perm + p + stride);
        }
        const V4<T> bv = window_gather(bulk4, x, valid, g, win);
        if (valid) {
            const DragOne<T> r = drag_from<T, EULER>(x, v, bv, g, P, dt);
            clamped_total += r.cl;
            F[p] = r.f[0];
            F[n + p] = r.f[1];
            F[2 * n + p] = r.f[2];
            st4(Fs, slot, r.f[0], r.f[1], r.f[2], T(0));
            st4(pos_out, slot, r.x[0], r.x[1], r.x[2], x.w);
            st4(vel_out, slot, r.u[0], r.u[1], r.u[2], v.w);
            drag_lane_sums(lane_sums, r);
        }
    }
    int wsum = clamped_total;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
    if ((threadIdx.x & 31) == 0 && wsum) {
        atomicAdd(&status[ST_CLAMPED], (unsigned long long)wsum);
        atomicOr(&status[ST_FLAGS], (unsigned long long)CG_FLAG_EPS_CLAMPED);
    }
    if (do_sums) {
        CSum<T> acc[kDragSums];
#pragma unroll
        for (int k = 0; k < kDragSums; ++k) acc[k].add(lane_sums[k]);
        block_sums<T, kDragSums>(acc, part, pstride, b.id);
    }
}

template <typename T, bool EULER>
__global__ void __launch_bounds__(256, 4)
k_drag_win(T* pos, T* vel, long long n, GridDev g, Phys<T> P, const T* __restrict__ bulk4, T* __restrict__ F,
           T* __restrict__ Fs, const int32_t* __restrict__ inv_perm, T dt, T* __restrict__ part, long long pstride,
           int do_sums, unsigned long long* __restrict__ status, T* __restrict__ pos_out, T* __restrict__ vel_out) {
    __shared__ __align__(16) V4<T> win[256 / 32][kWinRecs];
    pdl_wait();
    drag_body_win<T, EULER>(pos, vel, n, g, P, bulk4, F, Fs, inv_perm, dt, part, pstride, do_sums, status,
                            launch_blk(), pos_out, vel_out, win[threadIdx.x >> 5]);
}

template <typename T, bool EULER>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
k_drag(T* pos, T* vel, long long n, GridDev g, Phys<T> P, const T* __restrict__ bulk4,
       T* __restrict__ F, T* __restrict__ Fs, const int32_t* __restrict__ inv_perm, T dt,
       T* __restrict__ part, long long pstride, int do_sums, unsigned long long* __restrict__ status,
       T* __restrict__ Bs, T* __restrict__ pos_out, T* __restrict__ vel_out) {
    pdl_wait();
    drag_body<T, EULER>(pos, vel, n, g, P, bulk4, F, Fs, inv_perm, dt, part, pstride, do_sums, status,
                        launch_blk(), Bs, pos_out, vel_out);
}

// Batched drag with the fused sorted-order force record (FP32 instances).
template <bool EULER>
__global__ void __launch_bounds__(256) kb_drag(BLaunch L, float dt) {
    batch_loop(L, [&](const BInst& I, Blk b) {
        drag_body<float, EULER, false>(I.pos, I.vel, I.n, I.gd, I.P, I.bulk4, I.force, I.Fs, I.inv_perm, dt,
                                I.part + 2 * I.part_off[PS_DRAG], I.part_blocks[PS_DRAG], 1, I.status, b);
    });
}

cg_status launch_batch_drag(const BLaunch& L, unsigned grid, float dt, cudaStream_t s) {
    if (L.total == 0 || grid == 0) return CG_OK;
    if (dt > 0.f) kb_drag<true><<<grid, 256, 0, s>>>(L, dt);
    else kb_drag<false><<<grid, 256, 0, s>>>(L, 0.f);
    CG_CUDA(cudaGetLastError());
    return CG_OK;
}

int batch_drag_occupancy() {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_drag<true>, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return occ > 0 ? occ : 1;
}

cg_status launch_drag(cg_grids* g, long long n, const void* pos_d, const void* vel, void* force, void* S_bulk,
                      bool sums, double dt, void* coef_bulk, void* pos_out, void* vel_out) {
    const bool euler = dt > 0.0;
    void* part = part_ptr(g, PS_DRAG);
    // exactly the resident CTAs (the launch bounds' minimum per SM): a grid-stride
    // loop with no second, partial wave of blocks
    const long long per_sm = g->fp64 ? 2 : 4;
    const unsigned nblk = (unsigned)std::max(1LL, std::min((n + 255) / 256, (long long)g->num_sms * per_sm));
    g->part_blocks[PS_DRAG] = sums ? (long long)nblk : -1;
    void* Fs = S_bulk ? g->Fs : nullptr;
    if (pos_out && !Fs) return CG_ERR_INVALID_ARG;   // the sorted slots come with the fused reaction
    void* Bs = nullptr;
    if (coef_bulk && n > 0) {
        // sized by the step before its first launch
        if (g->Bs.bytes < 4 * g->tsize * (size_t)n) return CG_ERR_INVALID_ARG;
        Bs = g->Bs.p;
    }
    if (n > 0 || sums) {
#define CG_DRAGP(T, E)                                                                                      \
    CG_LAUNCH(g, "drag", (k_drag<T, E>), nblk, 256, 0, (T*)pos_d, (T*)vel, n, g->gd, phys_of<T>(g->gd),          \
              (const T*)g->bulk4, (T*)force, (T*)Fs, g->inv_perm, (T)dt, (T*)part, (long long)nblk, (int)sums,   \
              g->status, (T*)Bs, (T*)pos_out, (T*)vel_out)
        // on request, the sorted step (its particles come in nearly in cell
        // order) stages each warp's stencil window on the FP32 trilinear path
        const bool win = g->desc.stencil == CG_STENCIL_WINDOW && pos_out && !g->fp64 && !Bs &&
                         g->gd.interp != CG_INTERP_CELL;
        if (win) {
            if (euler)
                CG_LAUNCH(g, "drag", (k_drag_win<float, true>), nblk, 256, 0, (float*)pos_d, (float*)vel, n, g->gd,
                          phys_of<float>(g->gd), (const float*)g->bulk4, (float*)force, (float*)Fs, g->inv_perm,
                          (float)dt, (float*)part, (long long)nblk, (int)sums, g->status, (float*)pos_out,
                          (float*)vel_out);
            else
                CG_LAUNCH(g, "drag", (k_drag_win<float, false>), nblk, 256, 0, (float*)pos_d, (float*)vel, n, g->gd,
                          phys_of<float>(g->gd), (const float*)g->bulk4, (float*)force, (float*)Fs, g->inv_perm,
                          (float)dt, (float*)part, (long long)nblk, (int)sums, g->status, (float*)pos_out,
                          (float*)vel_out);
        } else if (g->fp64) {
            if (euler) CG_DRAGP(double, true);
            else CG_DRAGP(double, false);
        } else {
            if (euler) CG_DRAGP(float, true);
            else CG_DRAGP(float, false);
        }
#undef CG_DRAGP
    }
    if (S_bulk) CG_TRY(launch_deposit_sorted_force(g, n, S_bulk));
    if (coef_bulk) CG_TRY(launch_deposit_implicit(g, n, coef_bulk));
    return CG_OK;
}

}  // namespace cg
