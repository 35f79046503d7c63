// drag.cu -- (a3) drag on every particle, Eq. (DragLaw) of arXiv 1807.11834:
// F = beta (u_f - u_p), with the porosity and the fluid velocity taken at the
// particle from the bulk grid ("cell values or locally interpolated values",
// Sec. 1), and beta from a correlation of slip, densities, diameter,
// viscosity and porosity.  Optionally (a5) the semi-implicit Euler advance
// of Eq. (DEM_EQUATIONS) without contacts.
//
// One thread per particle in the caller's order: the particle record is
// read once (two 16-byte loads) and the force written once (three
// coalesced stores).  The bulk fields are gathered from a packed array of
// (phi, u_x, u_y, u_z) per cell, eight 16-byte loads that stay in L2.  For
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

namespace cg {

template <typename T> struct M;
template <> struct M<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ float log10_(float x) { return log10f(x); }
    static __device__ __forceinline__ float pi6() { return 0.52359877559829887f; }
    static __device__ __forceinline__ float pi8() { return 0.39269908169872415f; }
};
template <> struct M<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double log10_(double x) { return log10(x); }
    static __device__ __forceinline__ double pi6() { return 0.52359877559829887308; }
    static __device__ __forceinline__ double pi8() { return 0.39269908169872414817; }
};

template <typename T>
struct Phys {
    T rho, mu, rho_mu, eps_switch, eps_min, rho_p, g[3];
};

// ----------------------------------------------------------------------
// Interpolation weights on the bulk-centre lattice, per axis:
// xi = (x - x0)/H - 1/2, i0 = clamp(floor xi, 0, nb - 2), t = clamp(xi - i0, 0, 1).
// ----------------------------------------------------------------------
__device__ __forceinline__ void axis_weight(float x, const GridDev& g, int a, int& i0, float& t) {
    float s, e;
    two_sum(x, -g.x0h[a], s, e);
    e -= g.x0l[a];
    const float dh = s + e;
    const float dl = e - (dh - s);
    const float qh = dh * g.ihh[a];
    float ql = fmaf(dh, g.ihh[a], -qh);
    ql = fmaf(dh, g.ihl[a], ql);
    ql = fmaf(dl, g.ihh[a], ql);
    float xh, xl;
    two_sum(qh, -0.5f, xh, xl);
    xl += ql;
    float fi = floorf(xh);
    if (xh == fi && xl < 0.f) fi -= 1.f;
    const float top = (float)(g.nb[a] - 2);
    if (!(fi >= 0.f)) fi = 0.f;
    else if (fi > top) fi = top;
    i0 = (int)fi;
    float tt = (xh - fi) + xl;
    t = fminf(fmaxf(tt, 0.f), 1.f);
}

__device__ __forceinline__ void axis_weight(double x, const GridDev& g, int a, int& i0, double& t) {
    const double xi = __ddiv_rn(__dsub_rn(x, g.x0[a]), g.H[a]) - 0.5;
    double fi = floor(xi);
    const double top = (double)(g.nb[a] - 2);
    if (!(fi >= 0.0)) fi = 0.0;
    else if (fi > top) fi = top;
    i0 = (int)fi;
    t = fmin(fmax(xi - fi, 0.0), 1.0);
}

template <typename T>
__device__ __forceinline__ T lerp_(T a, T b, T t) { return fma(t, b - a, a); }

template <typename T>
__device__ __forceinline__ V4<T> lerp4(const V4<T>& a, const V4<T>& b, T t) {
    return {lerp_(a.x, b.x, t), lerp_(a.y, b.y, t), lerp_(a.z, b.z, t), lerp_(a.w, b.w, t)};
}

// Gather (phi, u) at a point.
template <typename T>
__device__ __forceinline__ V4<T> gather(const T* __restrict__ bulk4, T x, T y, T z, const GridDev& g) {
    if (g.interp == CG_INTERP_CELL) {
        int c = sizeof(T) == 4 ? cell_of_f((float)x, (float)y, (float)z, g)
                               : cell_of_d((double)x, (double)y, (double)z, g);
        return ld4(bulk4, c);
    }
    int i0, j0, k0;
    T tx, ty, tz;
    axis_weight(x, g, 0, i0, tx);
    axis_weight(y, g, 1, j0, ty);
    axis_weight(z, g, 2, k0, tz);
    const long long sx = 1, sy = g.nb[0], sz = (long long)g.nb[0] * g.nb[1];
    const long long c = i0 + sy * j0 + sz * k0;
    V4<T> a00 = lerp4(ld4(bulk4, c), ld4(bulk4, c + sx), tx);
    V4<T> a10 = lerp4(ld4(bulk4, c + sy), ld4(bulk4, c + sy + sx), tx);
    V4<T> a01 = lerp4(ld4(bulk4, c + sz), ld4(bulk4, c + sz + sx), tx);
    V4<T> a11 = lerp4(ld4(bulk4, c + sz + sy), ld4(bulk4, c + sz + sy + sx), tx);
    return lerp4(lerp4(a00, a10, ty), lerp4(a01, a11, ty), tz);
}

// ----------------------------------------------------------------------
// Per-particle drag factor beta_p (force = beta_p * slip).
//   eps: porosity seen by the law (already >= eps_min); phi = 1 - eps.
// Di Felice: 1/2 C_D0 rho (pi d^2/4) eps^2 |s| eps^-chi with
//   C_D0 |s| = (0.63 sqrt|s| + 4.8 / sqrt(rho eps d / mu))^2,
//   chi = 3.7 - 0.65 exp(-(1.5 - log10 Re)^2 / 2), Re = rho eps d |s| / mu.
// Ergun (eps < eps_switch): (150 phi mu / (eps d^2) + 1.75 rho |s| / d) V_p.
// Wen-Yu: 3/4 C_D |s| eps rho eps^-2.65 / d V_p with C_D |s| =
//   24 mu / (eps rho d) (1 + 0.15 (eps Re)^0.687) below eps Re = 1000, else 0.44 |s|.
// ----------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T drag_beta(int law, T eps, T phi, T d, T smag, const Phys<T>& P) {
    if (law == CG_DRAG_DI_FELICE) {
        const T red = P.rho_mu * eps * d;
        const T Re = red * smag;
        const T a = T(0.63) * M<T>::sqrt_(smag) + T(4.8) / M<T>::sqrt_(red);
        const T cds = a * a;
        T chi = T(3.7);
        if (Re > T(0)) {
            const T l = T(1.5) - M<T>::log10_(Re);
            chi = T(3.7) - T(0.65) * M<T>::exp_(T(-0.5) * l * l);
        }
        return M<T>::pi8() * P.rho * d * d * cds * M<T>::pow_(eps, T(2) - chi);
    }
    const T vp = M<T>::pi6() * d * d * d;
    if (eps < P.eps_switch) return (T(150) * phi * P.mu / (eps * d * d) + T(1.75) * P.rho * smag / d) * vp;
    const T eRe = eps * P.rho_mu * d * smag;
    T cds;
    if (eRe < T(1000)) cds = T(24) * P.mu / (eps * P.rho * d) * (T(1) + T(0.15) * M<T>::pow_(eRe, T(0.687)));
    else cds = T(0.44) * smag;
    return T(0.75) * cds * eps * P.rho * M<T>::pow_(eps, T(-2.65)) / d * vp;
}

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
// Drag kernel.  Partial sums (per block): V_p, F (3), |F|, m u (3), clamped.
// With EULER the particle is advanced in place after its force is known:
// u += dt (F/m + g), x += dt u, specular reflection at the domain faces.
// ----------------------------------------------------------------------
template <typename T, bool EULER>
__global__ void __launch_bounds__(256)
k_drag(T* pos, T* vel, long long n, GridDev g, Phys<T> P, const T* __restrict__ bulk4,
       T* __restrict__ F, T* __restrict__ Fs, const int32_t* __restrict__ inv_perm, T dt,
       T* __restrict__ part, long long pstride, int do_sums, unsigned long long* __restrict__ status) {
    T lane_sums[kDragSums];
#pragma unroll
    for (int k = 0; k < kDragSums; ++k) lane_sums[k] = T(0);
    int clamped_total = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const V4<T> x = EULER ? ld4_plain(pos, p) : ld4((const T*)pos, p);
        const V4<T> v = EULER ? ld4_plain(vel, p) : ld4((const T*)vel, p);
        const V4<T> b = gather(bulk4, x.x, x.y, x.z, g);
        T phi = b.x;
        T eps = T(1) - phi;
        int cl = 0;
        if (eps < P.eps_min) {
            eps = P.eps_min;
            phi = T(1) - P.eps_min;
            cl = 1;
        }
        clamped_total += cl;
        const T sx = b.y - v.x, sy = b.z - v.y, sz = b.w - v.z;
        const T smag = M<T>::sqrt_(sx * sx + sy * sy + sz * sz);
        const T d = x.w;
        const T beta = drag_beta(g.law, eps, phi, d, smag, P);
        const T fx = beta * sx, fy = beta * sy, fz = beta * sz;
        F[p] = fx;
        F[n + p] = fy;
        F[2 * n + p] = fz;
        if (Fs) st4(Fs, __ldg(inv_perm + p), fx, fy, fz, T(0));
        T ux = v.x, uy = v.y, uz = v.z;
        const T vp = M<T>::pi6() * d * d * d;
        const T m = P.rho_p * vp;
        if (EULER) {
            T xn[3] = {x.x, x.y, x.z};
            T un[3] = {v.x + dt * (fx / m + P.g[0]), v.y + dt * (fy / m + P.g[1]), v.z + dt * (fz / m + P.g[2])};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                T xa = xn[a] + dt * un[a];
                const T lo = (T)g.x0[a], hi = (T)g.xhi[a];
                if (xa < lo) { xa = T(2) * lo - xa; un[a] = -un[a]; }
                else if (xa > hi) { xa = T(2) * hi - xa; un[a] = -un[a]; }
                xn[a] = xa;
            }
            st4(pos, p, xn[0], xn[1], xn[2], d);
            st4(vel, p, un[0], un[1], un[2], v.w);
            ux = un[0];
            uy = un[1];
            uz = un[2];
        }
        lane_sums[0] += vp;
        lane_sums[1] += fx;
        lane_sums[2] += fy;
        lane_sums[3] += fz;
        lane_sums[4] += beta * smag;
        lane_sums[5] += m * ux;
        lane_sums[6] += m * uy;
        lane_sums[7] += m * uz;
        lane_sums[8] += (T)cl;
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
        block_sums<T, kDragSums>(acc, part, pstride);
    }
}

template <typename T>
static Phys<T> phys_of(const GridDev& g) {
    Phys<T> P;
    P.rho = (T)g.rho_f;
    P.mu = (T)g.mu_f;
    P.rho_mu = (T)(g.rho_f / g.mu_f);
    P.eps_switch = (T)g.eps_switch;
    P.eps_min = (T)g.eps_min;
    P.rho_p = (T)g.rho_p;
    for (int a = 0; a < 3; ++a) P.g[a] = (T)g.g[a];
    return P;
}

cg_status launch_drag(cg_grids* g, long long n, const void* pos_d, const void* vel, void* force, void* S_bulk,
                      bool sums, double dt) {
    const bool euler = dt > 0.0;
    void* part = part_ptr(g, PS_DRAG);
    const unsigned nblk = (unsigned)std::max(1LL, std::min((n + 255) / 256, (long long)g->num_sms * 8));
    g->part_blocks[PS_DRAG] = sums ? (long long)nblk : -1;
    void* Fs = S_bulk ? g->Fs : nullptr;
    if (n > 0 || sums) {
#define CG_DRAGP(T, E)                                                                                      \
    CG_LAUNCH(g, "drag", (k_drag<T, E>), nblk, 256, 0, (T*)pos_d, (T*)vel, n, g->gd, phys_of<T>(g->gd),          \
              (const T*)g->bulk4, (T*)force, (T*)Fs, g->inv_perm, (T)dt, (T*)part, (long long)nblk, (int)sums,   \
              g->status)
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
    return CG_OK;
}

}  // namespace cg
