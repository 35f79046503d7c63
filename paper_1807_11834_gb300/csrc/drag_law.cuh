// drag_law.cuh -- device pieces of the drag step shared by the plain and
// the learned drag kernels: interpolation weights on the bulk-centre
// lattice, the bulk-record gather, and the drag correlations of
// Eq. (DragLaw) of arXiv 1807.11834 (Di Felice; Ergun / Wen-Yu).
#pragma once

#include "cg_internal.cuh"

namespace cg {

// Math of the drag step.  The arithmetic of the correlations and of the
// Euler advance is written with explicitly rounded operations (mul, add,
// sub, div, and fma where a fused product is meant), so the compiler cannot
// fuse a product into an addition in one kernel and not in another: every
// kernel built from this code (plain, windowed, batched, learned) gives the
// same bits for the same particle.
template <typename T> struct M;
template <> struct M<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    // square root and reciprocal square root on the special-function unit
    // (sqrt.approx / rsqrt.approx: relative error about 2^-23, a rounding
    // or two; subnormal inputs count as 0, which turns a slip below 1e-19
    // into none, a drag that is zero to within 1e-19 of its scale anyway)
    static __device__ __forceinline__ float sqrt_(float x) {
        float y;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float rsqrt_(float x) {
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    // 1 / x on the special-function unit (rcp.approx: about one rounding; the
    // masses, porosities and diameters it divides by are normal numbers)
    static __device__ __forceinline__ float rcp_(float x) {
        float y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    // x^y for the correlations' bases, which are never negative (a porosity of
    // at least eps_min >= 0, or eps Re >= 0): 2^(y log2 x), without powf's
    // handling of negative bases and integer exponents; log2f (1 ulp) and
    // exp2f (2 ulp) keep the result within about 5e-7 relative for |y| < 3
    // and x in (0, 1000]; x = 0 gives 2^(-inf y), the same 0 or inf as powf
    static __device__ __forceinline__ float pow_(float x, float y) { return exp2f(__fmul_rn(y, log2f(x))); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    // log10 x = log2 x * log10 2 (log2f: 1 ulp)
    static __device__ __forceinline__ float log10_(float x) { return __fmul_rn(log2f(x), 0.30102999566398120f); }
    static __device__ __forceinline__ float pi6() { return 0.52359877559829887f; }
    static __device__ __forceinline__ float pi8() { return 0.39269908169872415f; }
};
template <> struct M<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double rsqrt_(double x) { return __ddiv_rn(1.0, sqrt(x)); }
    static __device__ __forceinline__ double rcp_(double x) { return __ddiv_rn(1.0, x); }
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
    // xi = x / H + xb as float-float: x * (1/H)_hi is exact as p + pe (FMA),
    // one TwoSum with xb_hi, the small terms added plainly (about 2^-44
    // relative to xi, as the float-float difference and product it replaces)
    const float p = __fmul_rn(x, g.ihh[a]);   // never fused into the TwoSum below
    const float pe = fmaf(x, g.ihh[a], -p);
    float xh, xl;
    two_sum(p, g.xbh[a], xh, xl);
    xl += pe + fmaf(x, g.ihl[a], g.xbl[a]);
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

// Read-only load of one packed record at p.
__device__ __forceinline__ V4<float> ldv4(const V4<float>* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ldv4(const V4<double>* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = __ldg(q), b = __ldg(q + 1);
    return {a.x, a.y, b.x, b.y};
}

template <typename T>
__device__ __forceinline__ V4<T> lerp4(const V4<T>& a, const V4<T>& b, T t) {
    return {lerp_(a.x, b.x, t), lerp_(a.y, b.y, t), lerp_(a.z, b.z, t), lerp_(a.w, b.w, t)};
}

// Trilinear value from the 8 records of a stencil: c the base corner,
// oy / oz the record steps along y / z (x is 1), read by ld; x, then y,
// then z, in this order wherever the records come from (global memory or a
// staged window), so every path gives the same value bit for bit.
template <typename T, typename Ld>
__device__ __forceinline__ V4<T> interp8(const V4<T>* c, int oy, int oz, T tx, T ty, T tz, Ld ld) {
    V4<T> a00 = lerp4(ld(c), ld(c + 1), tx);
    V4<T> a10 = lerp4(ld(c + oy), ld(c + oy + 1), tx);
    V4<T> a01 = lerp4(ld(c + oz), ld(c + oz + 1), tx);
    V4<T> a11 = lerp4(ld(c + oz + oy), ld(c + oz + oy + 1), tx);
    return lerp4(lerp4(a00, a10, ty), lerp4(a01, a11, ty), tz);
}

// Gather (eps, u) at a point.
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
    // cell indices fit in int (fewer than 2^31 bulk cells)
    const int sy = g.nb[0], sz = g.nb[0] * g.nb[1];
    return interp8<T>(reinterpret_cast<const V4<T>*>(bulk4) + (i0 + sy * j0 + sz * k0), sy, sz, tx, ty, tz,
                      [](const V4<T>* q) { return ldv4(q); });
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
    using X = M<T>;
    if (law == CG_DRAG_DI_FELICE) {
        const T red = X::mul(X::mul(P.rho_mu, eps), d);
        const T Re = X::mul(red, smag);
        const T a = X::fma_(T(0.63), X::sqrt_(smag), X::mul(T(4.8), X::rsqrt_(red)));
        const T cds = X::mul(a, a);
        T chi = T(3.7);
        if (Re > T(0)) {
            const T l = X::sub(T(1.5), X::log10_(Re));
            chi = X::fma_(T(-0.65), X::exp_(X::mul(X::mul(T(-0.5), l), l)), T(3.7));
        }
        return X::mul(X::mul(X::mul(X::mul(X::mul(X::pi8(), P.rho), d), d), cds), X::pow_(eps, X::sub(T(2), chi)));
    }
    const T vp = X::mul(X::mul(X::mul(X::pi6(), d), d), d);
    // Ergun (150 phi mu / (eps d^2) + 1.75 rho |s| / d) V_p with V_p = pi d^3 / 6,
    // rearranged to one division: pi/6 d (150 phi mu / eps + 1.75 rho |s| d)
    if (eps < P.eps_switch) {
        const T visc = X::mul(X::mul(X::mul(T(150), phi), P.mu), X::rcp_(eps));
        const T inert = X::mul(X::mul(X::mul(T(1.75), P.rho), smag), d);
        return X::mul(X::mul(X::pi6(), d), X::add(visc, inert));
    }
    const T eRe = X::mul(X::mul(X::mul(eps, P.rho_mu), d), smag);
    T cds;
    if (eRe < T(1000))
        cds = X::mul(X::mul(X::mul(T(24), P.mu), X::rcp_(X::mul(X::mul(eps, P.rho), d))),
                     X::fma_(T(0.15), X::pow_(eRe, T(0.687)), T(1)));
    else
        cds = X::mul(T(0.44), smag);
    return X::mul(X::mul(X::mul(X::mul(X::mul(X::mul(T(0.75), cds), eps), P.rho), X::pow_(eps, T(-2.65))),
                          X::rcp_(d)),
                  vp);
}

// Bulk record and its trilinear gradient at a point: eps, u (value) and
// d eps / dx_a (zero along an axis where the point is in the outer half
// cell, or in cell-value mode), plus an interpolated scalar field.
template <typename T>
struct Probe {
    T eps, ux, uy, uz, sc;
    T geps[3];
};

__device__ __forceinline__ bool axis_weight_cl(float x, const GridDev& g, int a, int& i0, float& t);
__device__ __forceinline__ bool axis_weight_cl(double x, const GridDev& g, int a, int& i0, double& t);

template <typename T>
__device__ __forceinline__ Probe<T> probe(const T* __restrict__ bulk4, const T* __restrict__ scal, T x, T y, T z,
                                          const GridDev& g) {
    Probe<T> r;
    if (g.interp == CG_INTERP_CELL) {
        const int c = sizeof(T) == 4 ? cell_of_f((float)x, (float)y, (float)z, g)
                                     : cell_of_d((double)x, (double)y, (double)z, g);
        const V4<T> b = ld4(bulk4, c);
        r.eps = b.x; r.ux = b.y; r.uy = b.z; r.uz = b.w;
        r.sc = scal ? __ldg(scal + c) : T(0);
        r.geps[0] = r.geps[1] = r.geps[2] = T(0);
        return r;
    }
    int i0, j0, k0;
    T tx, ty, tz;
    const bool cx = axis_weight_cl(x, g, 0, i0, tx);
    const bool cy = axis_weight_cl(y, g, 1, j0, ty);
    const bool cz = axis_weight_cl(z, g, 2, k0, tz);
    const long long sx = 1, sy = g.nb[0], sz = (long long)g.nb[0] * g.nb[1];
    const long long c = i0 + sy * j0 + sz * k0;
    const long long cc[8] = {c, c + sx, c + sy, c + sy + sx, c + sz, c + sz + sx, c + sz + sy, c + sz + sy + sx};
    V4<T> v[8];
    T s[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        v[q] = ld4(bulk4, cc[q]);
        s[q] = scal ? __ldg(scal + cc[q]) : T(0);
    }
    // value: x, then y, then z
    const V4<T> a00 = lerp4(v[0], v[1], tx), a10 = lerp4(v[2], v[3], tx);
    const V4<T> a01 = lerp4(v[4], v[5], tx), a11 = lerp4(v[6], v[7], tx);
    const V4<T> val = lerp4(lerp4(a00, a10, ty), lerp4(a01, a11, ty), tz);
    r.eps = val.x; r.ux = val.y; r.uy = val.z; r.uz = val.w;
    const T s00 = lerp_(s[0], s[1], tx), s10 = lerp_(s[2], s[3], tx);
    const T s01 = lerp_(s[4], s[5], tx), s11 = lerp_(s[6], s[7], tx);
    r.sc = lerp_(lerp_(s00, s10, ty), lerp_(s01, s11, ty), tz);
    // gradient of eps: difference along the axis, weights of the other two
    const T dx = lerp_(lerp_(v[1].x - v[0].x, v[3].x - v[2].x, ty), lerp_(v[5].x - v[4].x, v[7].x - v[6].x, ty), tz);
    const T dy = lerp_(lerp_(v[2].x - v[0].x, v[3].x - v[1].x, tx), lerp_(v[6].x - v[4].x, v[7].x - v[5].x, tx), tz);
    const T dz = lerp_(lerp_(v[4].x - v[0].x, v[5].x - v[1].x, tx), lerp_(v[6].x - v[2].x, v[7].x - v[3].x, tx), ty);
    r.geps[0] = cx ? T(0) : dx * (T)g.invH[0];
    r.geps[1] = cy ? T(0) : dy * (T)g.invH[1];
    r.geps[2] = cz ? T(0) : dz * (T)g.invH[2];
    return r;
}

// Axis weight with the clamp flag (the interpolant's gradient is zero
// along an axis where the point lies in the outer half cell).
__device__ __forceinline__ bool axis_weight_cl(float x, const GridDev& g, int a, int& i0, float& t) {
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
    const float tt = (xh - fi) + xl;
    t = fminf(fmaxf(tt, 0.f), 1.f);
    return !(tt >= 0.f && tt <= 1.f);
}
__device__ __forceinline__ bool axis_weight_cl(double x, const GridDev& g, int a, int& i0, double& t) {
    const double xi = __ddiv_rn(__dsub_rn(x, g.x0[a]), g.H[a]) - 0.5;
    double fi = floor(xi);
    const double top = (double)(g.nb[a] - 2);
    if (!(fi >= 0.0)) fi = 0.0;
    else if (fi > top) fi = top;
    i0 = (int)fi;
    const double tt = xi - fi;
    t = fmin(fmax(tt, 0.0), 1.0);
    return !(tt >= 0.0 && tt <= 1.0);
}

template <typename T>
inline Phys<T> phys_of(const GridDev& g) {
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

}  // namespace cg
