// cg_internal.cuh -- internal declarations of the GB300 coupling library.
//
// Shared by the .cu files of the library only (never by the oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/cg.h"

namespace cg {

// One-time settings that the CUDA runtime keeps per device (kernel
// attributes such as the dynamic shared-memory limit): f runs once on each
// device, the first time a call is made with that device current, under a
// lock; a failure is returned and retried on the next call.
struct PerDeviceOnce {
    std::mutex mu;
    bool done[64] = {};
};

template <typename F>
inline cg_status once_per_device(PerDeviceOnce& o, F f) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return CG_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(o.mu);
    if (o.done[dev]) return CG_OK;
    const cg_status s = f();
    if (s == CG_OK) o.done[dev] = true;
    return s;
}

// ----------------------------------------------------------------------
// Sizes
// ----------------------------------------------------------------------
constexpr int kSortThreads = 512;                   // threads of a sort tile
constexpr int kSortItems = 8;                       // items per thread
constexpr int kSortTile = kSortThreads * kSortItems; // 4096 particles per tile
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kMaxDigitBits = 11;                   // widest radix digit of one pass
constexpr int kMaxPasses = 3;
constexpr int kMaxBulkBits = 2 * kMaxDigitBits;     // two passes -> 2^22 cells
constexpr int kScanItems = 4096;                    // elements per scan block
// per-cell sort
constexpr int kKeyThreads = 256;                    // threads of its key kernel
constexpr int kKeyItems = 4;                        // particles per thread of the key kernel
constexpr int kPlaceItems = 4;                      // particles per thread of the placement
constexpr int kSegSortWarps = 8;                    // warps of a per-cell sort CTA
constexpr int kGroupCells = 8;                      // consecutive cells a warp takes at a time
constexpr int kWarpStage = 1024;                    // ids of a group staged in the warp's shared memory
constexpr int kSegWarpMax = 256;                    // largest cell a warp sorts in registers
// Split of a key of `bits` bits into the fewest passes of at most `digits`
// bits (at most kMaxPasses; wider only when the key needs it), the low
// digits first.  digits 0 takes the default: narrow digits (8) for grids of
// 2^20 cells and more, whose particles are usually far from cell order and
// whose scatters then profit from long digit runs (three passes measured
// faster on the 32M-particle clustered bed), wide ones (10) below (two
// passes measured faster on the 4M-particle packed bed).  Returns the passes.
inline int split_passes(int bits, int (&pb)[kMaxPasses], int digits = 0) {
    const int D = digits > 0 ? digits : (bits >= 20 ? 8 : 10);
    int np = (bits + D - 1) / D;
    np = np < 1 ? 1 : (np > kMaxPasses ? kMaxPasses : np);
    for (int i = 0; i < kMaxPasses; ++i) pb[i] = i < np ? bits / np + (i < bits % np ? 1 : 0) : 0;
    return np;
}

// cg_grid_desc.sort_digits: automatic, per-cell sort, or a digit width.
inline bool sort_choice_valid(int v) { return v == CG_SORT_AUTO || v == CG_SORT_CELLS || (v >= 6 && v <= kMaxDigitBits); }
// The per-cell sort serves a call of n particles over nbulk cells.
inline bool use_cell_sort(int v, long long n, long long nbulk) {
    return v == CG_SORT_CELLS ||
           (v == CG_SORT_AUTO && n <= CG_SORT_CELLS_AUTO_MAX && n <= (long long)CG_SORT_CELLS_AUTO_DENSITY * nbulk);
}

// Dynamic shared memory of a sort scatter pass with 2^bits digits: the
// per-warp counters, or the staged tile (key, id, diameter of T), whichever
// is larger, plus two [2^bits] int arrays.
__host__ __device__ constexpr size_t scatter_smem_bytes(int bits, size_t tsize) {
    return ((size_t)kSortWarps * sizeof(int) << bits) > (size_t)kSortTile * (8 + tsize)
               ? (((size_t)kSortWarps * sizeof(int) << bits) + (2 * sizeof(int) << bits))
               : ((size_t)kSortTile * (8 + tsize) + (2 * sizeof(int) << bits));
}
constexpr int kNumSlots = 16;                       // status counters

// Status word slots (unsigned long long each).
enum { ST_FLAGS = 0, ST_OUTSIDE = 1, ST_NONFINITE = 2, ST_CLAMPED = 3, ST_TIMEOUT = 4, ST_FALLBACK = 5 };

// Partial-sum regions of the conservation sums.
// The projection's region holds six columns: sum S_f V_f (3), then sum S_B
// V_B (3) of the source it reads.
enum { PS_VOL = 0, PS_DRAG = 1, PS_PROJ = 2, PS_NREG = 3 };
constexpr int kDragSums = 9;   // V_p, F(3), |F|, m u (3), clamped count
constexpr int kDragCellSums = kDragSums + 3;   // + S_B V_B (3) in the cell-order drag

// ----------------------------------------------------------------------
// Device-side view of the grid geometry (passed by value to kernels)
// ----------------------------------------------------------------------
struct GridDev {
    int nb[3];          // bulk cells per axis
    int nf[3];          // fine cells per axis
    int r;              // coarsening ratio
    long long nbulk, nfine;
    double x0[3];       // origin
    double xhi[3];      // origin + extent
    double H[3];        // bulk spacing (L / nb, rounded to double)
    double invH[3];     // 1 / H (double)
    double VB, invVB, Vf;
    // float versions for the FP32 path
    float x0f[3];       // (float)x0
    float xhif[3];      // (float)xhi
    float invHf[3];     // (float)(1/H)
    float ax0f[3];      // |x0 / H| (filter margin term)
    float x0h[3], x0l[3];   // x0 as float-float
    float ihh[3], ihl[3];   // 1/H as float-float
    float xbh[3], xbl[3];   // -(x0 / H + 1/2) as float-float: the lattice coordinate is x / H + xb
    float invVBf, VBf, Vff;
    float VBh, VBl, Vfh, Vfl;   // V_B, V_f as float-float
    float ivBh, ivBl;           // 1 / V_B as float-float
    // physics
    int law, interp;
    double rho_f, mu_f, rho_p, eps_switch, eps_min, g[3];
};

// ----------------------------------------------------------------------
// Handle
// ----------------------------------------------------------------------
struct ProfSlot {
    std::string name;
    long long launches = 0;
    double total_ms = 0.0;
};

struct PendingEv {
    int slot;
    int ev;   // index into the event pool (start = 2 ev, stop = 2 ev + 1)
};

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Device staging of one host-buffer step: inputs, outputs, and the events
// that order its copies and compute against the next use of the same set.
struct HostStage {
    DevBuf pos, vel, ufine, eps, ub, var, Sb, F, Sf, epsf, sums, cell, perm, cs;
    cudaEvent_t in_done = nullptr, comp_done = nullptr, out_done = nullptr;
    bool used = false;
};

}  // namespace cg

struct cg_grids {
    cg_grid_desc desc;
    cg::GridDev gd;
    int fp64 = 0;
    size_t tsize = 4;          // bytes of T
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 148;
    int bulk_bits = 0, pass_bits[cg::kMaxPasses] = {0, 0, 0}, npasses = 1;

    // binning state
    long long n_binned = -1;
    long long cap = -1;        // particle capacity of the particle buffers

    // particle-sized buffers
    int32_t* key = nullptr;        // [cap] cell per particle (caller order)
    int32_t* key1 = nullptr;       // [cap] keys after pass 1
    int32_t* val1 = nullptr;       // [cap] particle ids after pass 1
    int32_t* key2 = nullptr;       // [cap] keys after pass 2 of three
    int32_t* val2 = nullptr;       // [cap] particle ids after pass 2 of three
    int32_t* perm = nullptr;       // [cap] particle ids in cell order
    int32_t* key_sorted = nullptr; // [cap] cell of each slot of the sorted order
    int32_t* inv_perm = nullptr;   // [cap] sorted slot of each particle
    void* vol = nullptr;           // [cap] T particle diameter, caller order (for the volume deposit)
    void* vol_sorted = nullptr;    // [cap] T particle diameter, sorted order
    void* Fs = nullptr;            // [cap] T4 drag force, sorted order
    bool vol_valid = false;        // vol_sorted matches the binned positions
    bool key_valid = false;        // key holds the binning's caller-order cells (see ensure_keys)
    // incremental rebinning (rebin.cu): a binning of hint_n particles held in
    // perm / key_sorted / cell_start is where the next binning of the same
    // count starts; hint_ident is the particle array the last sorted step
    // wrote in that binning's order (so its particle i sat at old slot i)
    long long hint_n = -1;
    const void* hint_ident = nullptr;
    int32_t* rb_rid = nullptr;     // [cap] per old slot: its particle id (the caller's order kept)
    int32_t* rb_rkn = nullptr;     // [cap] per old slot: the new cell, complemented for a mover
    int2* rb_mov = nullptr;        // [rb_nblk * kRebinTile] movers, each block of old slots its own part: (id, cell | rank << 22)
    int2* rb_arr = nullptr;        // [cap] arrivals grouped by cell: (id, cell)
    int32_t* rb_small = nullptr;   // new counts / starts, arrivals, departures per cell; block movers; counters
    long long rb_nblk = 0;
    int32_t* hist = nullptr;       // [2^digit * ntiles]
    int32_t* scan_part = nullptr;  // scan block partials
    long long hist_cap = 0, scan_cap = 0;

    // bulk-sized buffers
    int32_t* cell_start = nullptr; // [nbulk + 1]
    void* bulk4 = nullptr;         // [nbulk] T4: eps, u_x, u_y, u_z
    void* eps_t = nullptr;         // [nbulk] T: porosity in the path precision
    void* partials = nullptr;      // conservation-sum block partials: (s, c) pairs of T
    long long part_off[cg::PS_NREG] = {0, 0, 0};
    long long part_blocks[cg::PS_NREG] = {0, 0, 0};
    long long part_cap = 0;
    double* sums_scratch = nullptr;   // [CG_NSUMS] when the caller gives none
    unsigned long long* status = nullptr;   // [kNumSlots]

    // host-buffer entries: two staging sets used in turn, and the copy
    // streams (inputs in, outputs out) that overlap consecutive steps
    cg::HostStage hs[2];
    int hs_next = 0;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    // the last host step that advanced its particles in place: the event
    // after their copies back and the host arrays they went to (a later
    // host step reading those arrays waits for them)
    cudaEvent_t part_out = nullptr;
    const void* part_pos = nullptr;
    const void* part_vel = nullptr;
    cg::DevBuf fresh4;   // [nbulk] T4: (phi, u) of the fresh field of cg_mlp_features
    cg::DevBuf Bs;       // [cap] T4: (beta, beta u) in sorted order, for the semi-implicit coefficients

    // second stream of the step: fine-grid work that does not depend on the
    // particle path runs beside it (fork / join through events)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_avg = nullptr, ev_pack = nullptr, ev_epsf = nullptr;

    // launch accounting / profiling
    long long launches = 0;
    bool prof = false;
    std::vector<cg::ProfSlot> slots;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<cg::PendingEv> pending;
    int ev_used = 0;
};

namespace cg {

// ----------------------------------------------------------------------
// Launch plumbing (api.cu)
// ----------------------------------------------------------------------
int prof_slot(cg_grids* g, const char* name);
void prof_begin(cg_grids* g, int slot, int* ev);
void prof_end(cg_grids* g, int slot, int ev);

// Launch a kernel on the handle's stream, count it, time it when profiling,
// and turn a launch error into CG_ERR_CUDA.
// Launches are programmatic dependent launches: the next kernel on the
// stream may be scheduled while this one drains, and every kernel launched
// here starts with pdl_wait(), which returns once the kernels it depends on
// have completed and their memory is visible (so each kernel still sees all
// earlier work; only the launch latency overlaps).
#define CG_LAUNCH(g, name, kernel, grid, block, smem, ...)                        \
    do {                                                                         \
        int slot_ = -1, ev_ = -1;                                                \
        if ((g)->prof) {                                                         \
            slot_ = cg::prof_slot((g), (name));                                  \
            cg::prof_begin((g), slot_, &ev_);                                    \
        }                                                                        \
        cudaLaunchAttribute a_[1];                                               \
        a_[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;           \
        a_[0].val.programmaticStreamSerializationAllowed = 1;                    \
        cudaLaunchConfig_t c_ = {};                                              \
        c_.gridDim = dim3((unsigned)(grid));                                     \
        c_.blockDim = dim3((unsigned)(block));                                   \
        c_.dynamicSmemBytes = (size_t)(smem);                                    \
        c_.stream = (g)->stream;                                                 \
        c_.attrs = a_;                                                           \
        c_.numAttrs = 1;                                                         \
        cudaError_t e_ = cudaLaunchKernelEx(&c_, kernel, __VA_ARGS__);           \
        (g)->launches++;                                                         \
        if (e_ == cudaSuccess) e_ = cudaGetLastError();                          \
        if ((g)->prof) cg::prof_end((g), slot_, ev_);                            \
        if (e_ != cudaSuccess) return CG_ERR_CUDA;                               \
    } while (0)

#define CG_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return CG_ERR_CUDA;      \
    } while (0)

#define CG_TRY(call)                                    \
    do {                                                \
        cg_status s_ = (call);                          \
        if (s_ != CG_OK) return s_;                     \
    } while (0)

// ----------------------------------------------------------------------
// Step launchers (one .cu each)
// ----------------------------------------------------------------------
// Up to three independent arrays are scanned by one pair of launches: blocks
// [0, n0) cover array 0, blocks [n0, n0 + n1) array 1, and so on.
constexpr int kScanArrays = 3;
struct ScanJob {
    const int32_t* in[kScanArrays] = {};
    int32_t* out[kScanArrays] = {};
    long long m[kScanArrays] = {};
    long long nblk[kScanArrays] = {};
    const int32_t* skip = nullptr;   // device flag: when 0, the outputs already hold the scans and nothing runs
};

// Column map of the conservation-sum reduction: sum k merges cnt[k]
// compensated pairs starting at pair off[k] of the partials.
struct SumsMap {
    long long off[CG_NSUMS];     // first pair of the partial column, -1 = not computed
    long long cnt[CG_NSUMS];     // number of partials
};

cg_status ensure_particle_capacity(cg_grids* g, long long n);
// Exclusive scans of up to kScanArrays int32 arrays (in[a] nullable: skipped).
cg_status scan_exclusive(cg_grids* g, int count, const int32_t* const* in, int32_t* const* out, const long long* m,
                         const int32_t* skip = nullptr);
// Placement and per-cell sort of the per-cell binning sort from the cell
// starts cs; with run_if set they do nothing unless *run_if != 0.
cg_status launch_cellsort_tail(cg_grids* g, long long n, const int32_t* cs, const int32_t* run_if);
// Incremental rebinning (rebin.cu).
constexpr int kRebinThreads = 256;
constexpr int kRebinItems = 4;
constexpr int kRebinTile = kRebinThreads * kRebinItems;   // old slots per block
constexpr int kRebinMaxArrivals = 256;                     // arrivals per cell before the fallback
constexpr int kRebinCounters = 8;
// The small rebinning arrays (three of n_b + 1 ints, one of nblk + 1, the
// counters) each start on a 256-byte boundary: the scan reads them as int4.
inline long long rebin_pad(long long ints) { return (ints + 63) / 64 * 64; }
inline long long rebin_small_ints(long long nbulk, long long nblk) {
    return 3 * rebin_pad(nbulk + 1) + rebin_pad(nblk + 1) + kRebinCounters;
}
// The binning of n particles from the handle's last binning of n; ident:
// the particles are that binning's sorted output (particle i at old slot i).
cg_status launch_rebin(cg_grids* g, long long n, const void* pos_d, bool ident, double* eps_fill, void* rec_fill,
                       void* eps_t_fill);
// g->key of the last binning (an identity-hint rebinning leaves it to be
// formed from its records on demand).
cg_status ensure_keys(cg_grids* g, long long n);
cg_status ensure_partials(cg_grids* g, long long n);

// eps_fill (nullable): also set this [n_b] porosity to 1 (when n > 0), and
// likewise the porosity of the drag record rec_fill and of eps_t_fill (T).
cg_status launch_bin(cg_grids* g, long long n, const void* pos_d, double* eps_fill = nullptr,
                     void* rec_fill = nullptr, void* eps_t_fill = nullptr);
// prefilled: eps already holds 1 for every cell (the binning set it);
// rec / eps_t (nullable, sorted-diameter path only): also write the porosity
// of occupied cells into the drag record and its T copy.
cg_status launch_deposit_volume(cg_grids* g, long long n, const void* pos_d, double* eps, bool sums,
                                bool prefilled = false, void* rec = nullptr, void* eps_t = nullptr);
cg_status launch_deposit_sorted_force(cg_grids* g, long long n, void* S_bulk);
// Gather the particle records into the binned order (cg_reorder_particles).
cg_status launch_reorder(cg_grids* g, long long n, const void* pos_d, const void* vel, void* pos_out, void* vel_out);
// Semi-implicit coefficients [4][n_b] (A, b) from the drag's sorted (beta, beta u) records.
cg_status launch_deposit_implicit(cg_grids* g, long long n, void* coef_bulk);
cg_status launch_deposit_momentum(cg_grids* g, long long n, const void* force_soa, void* S_bulk);
// rec (nullable): also write the mean velocity into the drag record's u part.
cg_status launch_average(cg_grids* g, const void* u_fine, void* u_bulk, void* var_bulk, void* rec = nullptr);
cg_status launch_pack(cg_grids* g, const double* eps, const void* u_bulk, bool want_eps_t);
// pos_out, vel_out (nullable, needs S_bulk): the particles, advanced when
// dt > 0, are written to these arrays in the order of the binning.
cg_status launch_drag(cg_grids* g, long long n, const void* pos_d, const void* vel, void* force, void* S_bulk,
                      bool sums, double dt, void* coef_bulk = nullptr, void* pos_out = nullptr,
                      void* vel_out = nullptr);
// Learned drag (FP32 only): bulk4 must hold (phi of this step, stale u).
cg_status launch_drag_learned(cg_grids* g, const cg_mlp* m, long long n, void* pos_d, void* vel,
                              const void* var_stale, const void* u_fine, int32_t age, void* force, void* S_bulk,
                              double dt);
cg_status grow_buf(DevBuf& b, size_t bytes);
// The closure's feature box (CG_MLP_NFEAT values each).
cg_status mlp_feature_box(const cg_mlp* m, float* lo, float* hi);
// The stale variance field, fine velocity and record age bound to a closure by cg_mlp_bind.
cg_status mlp_bound_inputs(const cg_mlp* m, const void** var_stale, const void** u_fine, int32_t* age);
cg_status launch_project(cg_grids* g, int ncomp, const void* const* in, void* const* out, bool sums);
cg_status launch_sums(cg_grids* g, double* sums);
// Sum columns of the partial regions (offsets in pairs; blocks < 0: region not formed).
SumsMap sums_map(const long long* part_off, const long long* part_blocks);
// First element (in units of T) of the partial region r.
inline void* part_ptr(cg_grids* g, int r) { return (char*)g->partials + 2 * g->tsize * g->part_off[r]; }

}  // namespace cg

// ----------------------------------------------------------------------
// Device helpers
// ----------------------------------------------------------------------
namespace cg {

template <typename T> struct V4;
template <> struct V4<float> {
    float x, y, z, w;
};
template <> struct V4<double> {
    double x, y, z, w;
};

__device__ __forceinline__ V4<float> ld4(const float* __restrict__ p, long long i) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ld4(const double* __restrict__ p, long long i) {
    const double2* q = reinterpret_cast<const double2*>(p) + 2 * i;
    double2 a = __ldg(q), b = __ldg(q + 1);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st4(float* p, long long i, float x, float y, float z, float w) {
    reinterpret_cast<float4*>(p)[i] = make_float4(x, y, z, w);
}
__device__ __forceinline__ void st4(double* p, long long i, double x, double y, double z, double w) {
    double2* q = reinterpret_cast<double2*>(p) + 2 * i;
    q[0] = make_double2(x, y);
    q[1] = make_double2(z, w);
}

// Knuth's TwoSum: s + e == a + b exactly.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e) {
    s = a + b;
    T z = s - a;
    e = (a - (s - z)) + (b - z);
}

// A float's exact value as a double, assembled from its bits with integer
// operations (sign, exponent rebiased by 1023 - 127, mantissa shifted to the
// double's 52 bits), so that no conversion instruction lands on the FP64
// pipe; subnormal floats (below 2^-126) take the ordinary conversion.
__device__ __forceinline__ double f32_exact_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u && (u & 0x7fffffu)) return (double)f;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const unsigned long long ex = e == 0u ? 0ull : e == 255u ? 0x7ffull << 52 : (unsigned long long)(e + 896u) << 52;
    const unsigned long long man = (unsigned long long)(u & 0x7fffffu) << 29;
    return __longlong_as_double((long long)(sign | ex | man));
}

// Porosity 1 - V / V_B of a bulk cell from its compensated volume sum
// V = s + c: as a double (the output) and in the working precision (the
// drag's record and the porosity projection).  FP32 path: the product with
// 1 / V_B and the difference in float-float (relative error about 2^-46 of
// V / V_B, the accuracy of the volume sum itself), then one FP64 addition
// of the exact pair (GB300 issues FP64 at 1/64 of the FP32 rate, and this
// runs wherever a lane of the warp closes a cell); FP64 path: plain double
// arithmetic.
__device__ __forceinline__ void cell_porosity(float s, float c, const GridDev& g, double& e, float& et) {
    const float ph = s * g.ivBh;
    float pl = fmaf(s, g.ivBh, -ph);   // s / V_B = ph + pl to second order
    pl = fmaf(s, g.ivBl, pl);
    pl = fmaf(c, g.ivBh, pl);
    float eh, el;
    two_sum(1.0f, -ph, eh, el);
    el -= pl;
    float hi, lo;
    two_sum(eh, el, hi, lo);
    e = f32_exact_f64(hi) + f32_exact_f64(lo);
    et = hi;
}
__device__ __forceinline__ void cell_porosity(double s, double c, const GridDev& g, double& e, double& et) {
    e = 1.0 - (s + c) * g.invVB;
    et = e;
}

// Compensated accumulator (TwoSum cascade, Neumaier-equivalent).
template <typename T>
struct CSum {
    T s = T(0), c = T(0);
    __device__ __forceinline__ void add(T x) {
        T t, e;
        two_sum(s, x, t, e);
        s = t;
        c += e;
    }
    __device__ __forceinline__ void merge(const CSum& o) {
        add(o.s);
        c += o.c;
    }
    __device__ __forceinline__ T get() const { return s + c; }
};

// Warp-level fixed-tree reduction of a compensated sum (deterministic).
template <typename T>
__device__ __forceinline__ CSum<T> warp_reduce(CSum<T> v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        CSum<T> o;
        o.s = __shfl_xor_sync(0xffffffffu, v.s, off);
        o.c = __shfl_xor_sync(0xffffffffu, v.c, off);
        v.merge(o);
    }
    return v;
}

// Block coordinates of a kernel body: the launch's own (blockIdx.x,
// gridDim.x) for one instance, or a virtual block of one instance inside a
// batched launch over many instances.
struct Blk {
    long long id;   // block index within the instance's work
    long long n;    // number of blocks of the instance's work
};
__device__ __forceinline__ Blk launch_blk() { return {(long long)blockIdx.x, (long long)gridDim.x}; }

// Block-level deterministic reduction of K compensated sums.  Thread 0..K-1
// writes the pair (s, c) of sum k to part[2 * (k * stride + bid)]:
// partials stay in the path precision as compensated pairs, so no FP64
// arithmetic runs per block (GB300's FP64 rate is a small fraction of FP32).
template <typename T, int K>
__device__ __forceinline__ void block_sums(CSum<T> (&v)[K], T* __restrict__ part, long long stride, long long bid) {
    __shared__ T sh_s[K][32];
    __shared__ T sh_c[K][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        CSum<T> r = warp_reduce(v[k]);
        if (lane == 0) {
            sh_s[k][warp] = r.s;
            sh_c[k][warp] = r.c;
        }
    }
    __syncthreads();
    if (threadIdx.x < K) {
        const int k = threadIdx.x;
        CSum<T> a;
        a.s = sh_s[k][0];
        a.c = sh_c[k][0];
        for (int w = 1; w < nw; ++w) {
            CSum<T> o;
            o.s = sh_s[k][w];
            o.c = sh_c[k][w];
            a.merge(o);
        }
        T* dst = part + 2 * ((long long)k * stride + bid);
        dst[0] = a.s;
        dst[1] = a.c;
    }
}

// Block-wide exclusive scan of one int per thread (total in `total`); every
// thread of the block must call it.
__device__ __forceinline__ int block_exclusive_scan(int v, int* sh_warp, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) sh_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? sh_warp[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        sh_warp[lane] = w;   // inclusive warp totals
    }
    __syncthreads();
    int wbase = warp ? sh_warp[warp - 1] : 0;
    total = sh_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return wbase + x - v;
}

// Length of the run of equal values starting at this lane, or 0 if the lane
// is not the first of its run (runs of consecutive lanes with equal v).
__device__ __forceinline__ int run_head_length(int v, bool valid) {
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, v, 1);
    const bool head = valid && (lane == 0 || prev != v);
    const unsigned heads = __ballot_sync(0xffffffffu, head) | __ballot_sync(0xffffffffu, !valid);
    if (!head) return 0;
    const unsigned later = heads & ~((2u << lane) - 1u);
    const int next = lane == 31 ? 32 : (later ? __ffs(later) - 1 : 32);
    return next - lane;
}

// Programmatic dependent launch: wait until the grids this one depends on
// have completed and flushed their memory (returns at once for a kernel not
// launched as a dependent).  First statement of every kernel of the
// library (required of those launched through CG_LAUNCH).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ----------------------------------------------------------------------
// (a0) bin index, shared by the binning and the cell-value gather.
// ----------------------------------------------------------------------
// ----------------------------------------------------------------------
__device__ __forceinline__ int bin_axis_exact(double x, double x0, double H, int nb, int& outside) {
    double q = __ddiv_rn(__dsub_rn(x, x0), H);
    int i;
    if (!(q >= 0.0)) i = 0;
    else if (q >= (double)nb) i = nb - 1;
    else i = (int)floor(q);
    if (!(q >= 0.0 && q <= (double)nb)) outside = 1;
    return i;
}

// |q32 - q64| <= 4 u (|q| + |x0/H|), u = 2^-24, for
// q32 = (x - fl(x0)) * fl(1/H) in round-to-nearest float; the margin below
// is twice that bound.  Outside the margin floor(q32) == floor(q64).
__device__ __forceinline__ int bin_axis_f32(float x, const GridDev& g, int a, int& outside) {
    float q = __fmul_rn(__fsub_rn(x, g.x0f[a]), g.invHf[a]);
    float fl = floorf(q);
    float m = (fabsf(q) + g.ax0f[a]) * 4.76837158203125e-7f + 1e-30f;
    if ((q - fl > m) && (fl + 1.0f - q > m)) {
        int i = (int)fl;
        if (i < 0) { outside = 1; return 0; }
        if (i >= g.nb[a]) { outside = 1; return g.nb[a] - 1; }
        return i;
    }
    return bin_axis_exact((double)x, g.x0[a], g.H[a], g.nb[a], outside);
}

__device__ __forceinline__ int cell_of(const V4<float>& v, const GridDev& g, int& outside) {
    int i = bin_axis_f32(v.x, g, 0, outside);
    int j = bin_axis_f32(v.y, g, 1, outside);
    int k = bin_axis_f32(v.z, g, 2, outside);
    return i + g.nb[0] * (j + g.nb[1] * k);
}
__device__ __forceinline__ int cell_of(const V4<double>& v, const GridDev& g, int& outside) {
    int i = bin_axis_exact(v.x, g.x0[0], g.H[0], g.nb[0], outside);
    int j = bin_axis_exact(v.y, g.x0[1], g.H[1], g.nb[1], outside);
    int k = bin_axis_exact(v.z, g.x0[2], g.H[2], g.nb[2], outside);
    return i + g.nb[0] * (j + g.nb[1] * k);
}

__device__ __forceinline__ int cell_of_f(float x, float y, float z, const GridDev& g) {
    int o = 0;
    return cell_of(V4<float>{x, y, z, 0.f}, g, o);
}
__device__ __forceinline__ int cell_of_d(double x, double y, double z, const GridDev& g) {
    int o = 0;
    return cell_of(V4<double>{x, y, z, 0.0}, g, o);
}

// ----------------------------------------------------------------------
// Segmented reductions over the sorted particle order.
//
// The sorted order is cut into chunks of kSegChunk slots; warp w owns the
// segments (cells) that START in its chunks and runs past a chunk's end to
// finish its last segment, so every segment is reduced by exactly one warp
// and the work follows the particles, not the cells (a dense bed occupying
// a few percent of the cells still spreads over every SM).  The warp reduces
// its range in rounds: 32 slots a round, one per lane, with a segmented
// shuffle scan (seg_rounds: the reaction), or 256 slots a round, 8
// consecutive ones per lane (seg_seq: the porosity).  The rounds start at the
// range's first slot, so the summation order depends only on the chunk's
// slots, never on the launch shape.
// ----------------------------------------------------------------------
constexpr int kSegChunk = 256;

// Range [s, t) of sorted slots owned by the chunk starting at `base`.
__device__ __forceinline__ void seg_chunk_range(long long base, long long n, const int32_t* __restrict__ key_sorted,
                                                const int32_t* __restrict__ cs, long long& s, long long& t) {
    const long long last = (base + kSegChunk < n ? base + kSegChunk : n) - 1;
    s = base;
    if (base > 0) {
        const int k0 = __ldg(key_sorted + base);
        if (__ldg(key_sorted + base - 1) == k0) s = __ldg(cs + k0 + 1);
    }
    t = __ldg(cs + __ldg(key_sorted + last) + 1);
    if (s > last) t = s;   // the whole chunk lies inside a segment owned earlier
}

// Segmented sum of K values per slot over the slots [s, t) of one chunk,
// 32 slots per round: a plain shuffle scan inside the round (at most five
// roundings), compensated sums for the carry between rounds and for each
// segment's total.  load(i, v) fills the K values of slot i; emit(key, tot)
// receives each segment's compensated total on the lane of its last slot.
// The next round's slots are loaded before the current one is reduced.
template <typename T, int K, typename Load, typename Emit>
__device__ __forceinline__ void seg_rounds(long long s, long long t, const int32_t* __restrict__ key_sorted,
                                           Load load, Emit emit) {
    constexpr int B = 4;   // rounds loaded ahead of the reduction
    const int lane = threadIdx.x & 31;
    CSum<T> carry[K];
    int carry_key = -1;
    for (long long r0 = s; r0 < t; r0 += 32 * B) {
        int key[B + 1];
        T v[B][K];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const long long i = r0 + 32 * j + lane;
            key[j] = -1;
#pragma unroll
            for (int k = 0; k < K; ++k) v[j][k] = T(0);
            if (i < t) {
                key[j] = __ldg(key_sorted + i);
                load(i, v[j]);
            }
        }
        {
            const long long i = r0 + 32 * B + lane;
            key[B] = (lane == 0 && i < t) ? __ldg(key_sorted + i) : -1;   // first key after the batch
        }
#pragma unroll
        for (int j = 0; j < B; ++j) {
            if (r0 + 32 * j >= t) break;   // warp-uniform
            const long long i = r0 + 32 * j + lane;
            const bool valid = i < t;
            const int kj = key[j];
            T* vj = v[j];
            // plain inclusive segmented scan over the lanes
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int ko = __shfl_up_sync(0xffffffffu, kj, off);
                const bool take = lane >= off && ko == kj;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const T vo = __shfl_up_sync(0xffffffffu, vj[k], off);
                    if (take) vj[k] += vo;
                }
            }
            // every lane takes part in both shuffles; lane 31 looks at the next round
            int next = __shfl_down_sync(0xffffffffu, kj, 1);
            const int next31 = __shfl_sync(0xffffffffu, j + 1 < B ? key[j + 1] : key[B], 0);
            if (lane == 31) next = next31;
            const bool ends = valid && next != kj;
            const bool cont = kj == carry_key;
            if (ends) {
                CSum<T> tot[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if (cont) tot[k] = carry[k];
                    tot[k].add(vj[k]);
                }
                emit(kj, tot);
            }
            // carry: the segment of lane 31 if it goes on into the next round
            const int k31 = __shfl_sync(0xffffffffu, kj, 31);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const T v31 = __shfl_sync(0xffffffffu, vj[k], 31);
                if (k31 != carry_key) carry[k] = CSum<T>();
                carry[k].add(v31);
            }
            carry_key = k31;
        }
    }
}

// Segmented sums over the slots [s, t) of one chunk, 256 slots per round.
// Lane l walks its own 8 consecutive slots r0 + 8l .. r0 + 8l + 7 in order
// with compensated sums: runs that start and end inside the lane are
// emitted at once; the open first and last runs of the lanes are joined by
// one segmented scan over the lanes (compensated merges, lower slots
// first), and the round's last run is carried into the next round.  With
// EXACT every addition is compensated; otherwise a lane adds its own (at
// most 8) slots plainly and only the joins are compensated.  load(i, v)
// fills slot i's K compensated values; emit(key, tot) receives each
// segment's total (on one lane, once).  The summation order depends only on
// the chunk's slots, not on the launch.
template <typename T, int K, bool EXACT, typename Load, typename Emit>
__device__ __forceinline__ void seg_seq(long long s, long long t, const int32_t* __restrict__ key_sorted,
                                        Load load, Emit emit) {
    constexpr int P = 8;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    CSum<T> carry[K];
    int carry_key = -1;
    for (long long r0 = s; r0 < t; r0 += 32 * P) {
        const long long b0 = r0 + (long long)P * lane;
        int key[P];
        CSum<T> v[P][K];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            key[j] = -1;
            if (b0 + j < t) {
                key[j] = __ldg(key_sorted + b0 + j);
                load(b0 + j, v[j]);
            }
        }
        const int nk = (r0 + 32 * P < t) ? __ldg(key_sorted + r0 + 32 * P) : -1;   // first key after the round
        // the lane's own slots: head run, complete middle runs, open tail run
        const int head_key = key[0];
        int cur = key[0];
        int nruns = key[0] >= 0 ? 1 : 0;
        CSum<T> acc[K], head[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = v[0][k];
#pragma unroll
        for (int j = 1; j < P; ++j) {
            if (key[j] < 0) break;
            if (key[j] != cur) {
                if (nruns == 1) {
#pragma unroll
                    for (int k = 0; k < K; ++k) head[k] = acc[k];
                } else {
                    emit(cur, acc);
                }
                ++nruns;
                cur = key[j];
#pragma unroll
                for (int k = 0; k < K; ++k) acc[k] = v[j][k];
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if (EXACT) acc[k].merge(v[j][k]);
                    else acc[k].s += v[j][k].s;
                }
            }
        }
        const int tail_key = nruns ? cur : -2;
        // lane 0 continues the run carried from the previous round
        if (lane == 0 && nruns == 1 && head_key == carry_key)
#pragma unroll
            for (int k = 0; k < K; ++k) {
                CSum<T> c0 = carry[k];
                c0.merge(acc[k]);
                acc[k] = c0;
            }
        // segmented inclusive scan of the tail runs over the lanes: a lane
        // holding one run of the previous lane's tail key continues it
        const int prev_tail = __shfl_up_sync(full, tail_key, 1);
        bool fl = lane == 0 || nruns != 1 || head_key != prev_tail;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const bool ofl = __shfl_up_sync(full, fl, off);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                CSum<T> o;
                o.s = __shfl_up_sync(full, acc[k].s, off);
                o.c = __shfl_up_sync(full, acc[k].c, off);
                if (lane >= off && !fl) {
                    o.merge(acc[k]);
                    acc[k] = o;
                }
            }
            if (lane >= off && !fl) fl = ofl;
        }
        // head runs that end inside a lane take the chain before them
        CSum<T> before[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            before[k].s = __shfl_up_sync(full, acc[k].s, 1);
            before[k].c = __shfl_up_sync(full, acc[k].c, 1);
        }
        if (nruns > 1) {
            CSum<T> tot[K];
            const bool cont = lane == 0 ? head_key == carry_key : head_key == prev_tail;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                tot[k] = cont ? (lane == 0 ? carry[k] : before[k]) : CSum<T>();
                tot[k].merge(head[k]);
            }
            emit(head_key, tot);
        }
        // tail runs that end at the lane's end
        int next = __shfl_down_sync(full, head_key, 1);
        if (lane == 31) next = nk;
        const int last = (int)min((long long)31, (t - r0 - 1) / P);   // last lane holding slots
        if (lane == last) next = nk;
        if (nruns > 0 && next != tail_key) emit(tail_key, acc);
        // carry the round's last run into the next round
        const int lk = __shfl_sync(full, tail_key, last);
        const bool goes_on = nk >= 0 && nk == lk;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            carry[k].s = __shfl_sync(full, acc[k].s, last);
            carry[k].c = __shfl_sync(full, acc[k].c, last);
        }
        carry_key = goes_on ? lk : -1;
    }
}

// Reaction of one cell from its compensated force sum a: S_B = -(1/V_B) sum F
// (Eq. UFP: F_fpi is the fluid-side reaction to F_drag), written to S
// ([3][n_b]).  The conservation sum of S_B V_B is formed by the projection,
// which reads every S_B.
template <typename T>
__device__ __forceinline__ void reaction_emit(const GridDev& g, T* __restrict__ S, int key, const CSum<T> (&a)[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T s_;
        if (sizeof(T) == 4) s_ = -(a[k].get()) * (T)g.invVBf;
        else s_ = -(a[k].get()) * (T)g.invVB;
        S[k * g.nbulk + key] = s_;
    }
}

// Sphere volume pi d^3 / 6 as an unevaluated pair hi + lo: exact products
// by FMA in FP32 (relative error ~2^-46), the plain product in FP64.
__device__ __forceinline__ void sphere_volume_pair(float d, float& hi, float& lo) {
    const float p = d * d;
    const float pe = fmaf(d, d, -p);             // d^2 = p + pe exactly
    const float q = p * d;
    const float qe = fmaf(p, d, -q);             // p d = q + qe exactly
    const float r = fmaf(pe, d, qe);             // d^3 = q + r (to 2^-48)
    const float ch = 0.5235987901687622f;        // pi / 6 = ch + cl
    const float cl = -1.457046305830545e-08f;
    hi = ch * q;
    const float he = fmaf(ch, q, -hi);
    lo = fmaf(ch, r, fmaf(cl, q, he));
}
__device__ __forceinline__ void sphere_volume_pair(double d, double& hi, double& lo) {
    hi = 0.52359877559829887308 * d * d * d;
    lo = 0.0;
}

// Inclusive segmented scan of K compensated sums over the lanes, keyed by
// `key`; lane i ends with the sum of its segment's lanes <= i.
template <typename T, int K>
__device__ __forceinline__ void warp_seg_scan(CSum<T> (&v)[K], int key) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int ko = __shfl_up_sync(0xffffffffu, key, off);
        const bool take = lane >= off && ko == key;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            CSum<T> o;
            o.s = __shfl_up_sync(0xffffffffu, v[k].s, off);
            o.c = __shfl_up_sync(0xffffffffu, v[k].c, off);
            if (take) {
                // earlier lanes first: result = o (+) v
                CSum<T> r = o;
                r.merge(v[k]);
                v[k] = r;
            }
        }
    }
}

}  // namespace cg
