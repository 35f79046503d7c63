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
// float-float (TwoSum / FMA TwoProduct), so the interpolation weights carry
// only the final float rounding even at |xi| ~ 100; the correlations run in
// float with IEEE division and square root.
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
__device__ __forceinline__ DragOne<T> drag_one(const V4<T>& x, const V4<T>& v, const GridDev& g, const Phys<T>& P,
                                               const T* __restrict__ bulk4, T dt) {
    DragOne<T> r;
    const V4<T> b = gather(bulk4, x.x, x.y, x.z, g);
    T eps = b.x;
    T phi = T(1) - eps;
    r.cl = 0;
    if (eps < P.eps_min) {
        eps = P.eps_min;
        phi = T(1) - P.eps_min;
        r.cl = 1;
    }
    const T sx = b.y - v.x, sy = b.z - v.y, sz = b.w - v.z;
    r.smag = M<T>::sqrt_(sx * sx + sy * sy + sz * sz);
    const T d = x.w;
    r.beta = drag_beta(g.law, eps, phi, d, r.smag, P);
    r.f[0] = r.beta * sx;
    r.f[1] = r.beta * sy;
    r.f[2] = r.beta * sz;
    r.vp = M<T>::pi6() * d * d * d;
    r.m = P.rho_p * r.vp;
    r.x[0] = x.x;
    r.x[1] = x.y;
    r.x[2] = x.z;
    r.u[0] = v.x;
    r.u[1] = v.y;
    r.u[2] = v.z;
    if (EULER) {
        const T inv_m = T(1) / r.m;   // one division for the three components
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            T ua = r.u[a] + dt * (r.f[a] * inv_m + P.g[a]);
            T xa = r.x[a] + dt * ua;
            // the FP32 path reads the bounds' float copies (no conversion in the loop)
            const T lo = sizeof(T) == 4 ? (T)g.x0f[a] : (T)g.x0[a];
            const T hi = sizeof(T) == 4 ? (T)g.xhif[a] : (T)g.xhi[a];
            if (xa < lo) { xa = T(2) * lo - xa; ua = -ua; }
            else if (xa > hi) { xa = T(2) * hi - xa; ua = -ua; }
            r.x[a] = xa;
            r.u[a] = ua;
        }
    }
    return r;
}

// Per-lane diagnostics: V_p, F (3), |F|, m u (3) after the advance, clamped.
template <typename T>
__device__ __forceinline__ void drag_lane_sums(T (&ls)[kDragSums], const DragOne<T>& r) {
    ls[0] += r.vp;
    ls[1] += r.f[0];
    ls[2] += r.f[1];
    ls[3] += r.f[2];
    ls[4] += r.beta * r.smag;
    ls[5] += r.m * r.u[0];
    ls[6] += r.m * r.u[1];
    ls[7] += r.m * r.u[2];
    ls[8] += (T)r.cl;
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
        if (g->fp64) {
            if (euler) CG_DRAGP(double, true);
            else CG_DRAGP(double, false);
        } else {
            if (euler) CG_DRAGP(float, true);
            else CG_DRAGP(float, false);
        }
#undef CG_DRAGP
    }
    if (S_bulk) CG_TRY(launch_deposit_sorted_force(g, n, S_bulk, sums));
    if (coef_bulk) CG_TRY(launch_deposit_implicit(g, n, coef_bulk));
    return CG_OK;
}

}  // namespace cg
