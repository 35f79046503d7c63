// api.cu -- the C ABI of include/cg.h: argument checks, handle and buffer
// management, and the orchestration of the coupling step on one stream.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>

#include "cg_internal.cuh"

using namespace cg;

namespace {

bool finite3(const double* v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Host-side fault injection (cg_debug_fail_alloc_after): the number of
// handle-owned allocations still allowed before one fails; -1 = none fails.
std::atomic<long long> g_alloc_fail_after{-1};

bool injected_alloc_failure() {
    long long k = g_alloc_fail_after.load();
    while (k >= 0)
        if (g_alloc_fail_after.compare_exchange_weak(k, k - 1)) return k == 0;   // after the failure: -1
    return false;
}

template <typename P>
cg_status dalloc(P** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (injected_alloc_failure()) return CG_ERR_OOM;
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? CG_ERR_OOM : CG_ERR_CUDA;
    }
    *p = (P*)q;
    return CG_OK;
}

template <typename P>
void dfree(P*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

cg_status ensure_buf(DevBuf& b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return CG_OK;
    dfree(b.p);
    b.bytes = 0;
    CG_TRY(dalloc(&b.p, bytes));
    b.bytes = bytes;
    return CG_OK;
}

void split_ff(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

int ceil_log2(long long v) {
    int b = 0;
    while ((1LL << b) < v) ++b;
    return b;
}

cg_status check_handle(const cg_grids* g) { return g ? CG_OK : CG_ERR_INVALID_ARG; }

}  // namespace

namespace cg {

cg_status grow_buf(DevBuf& b, size_t bytes) { return ensure_buf(b, bytes); }

// ---------------------------------------------------------------------------
// Profiling plumbing
// ---------------------------------------------------------------------------
int prof_slot(cg_grids* g, const char* name) {
    for (size_t i = 0; i < g->slots.size(); ++i)
        if (g->slots[i].name == name) return (int)i;
    ProfSlot s;
    s.name = name;
    g->slots.push_back(s);
    return (int)g->slots.size() - 1;
}

static void prof_drain(cg_grids* g) {
    if (g->pending.empty()) return;
    cudaStreamSynchronize(g->stream);
    for (const PendingEv& pe : g->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g->ev_pool[2 * pe.ev], g->ev_pool[2 * pe.ev + 1]) == cudaSuccess) {
            g->slots[pe.slot].total_ms += ms;
            g->slots[pe.slot].launches += 1;
        }
    }
    cudaGetLastError();
    g->pending.clear();
    g->ev_used = 0;
}

void prof_begin(cg_grids* g, int slot, int* ev) {
    (void)slot;
    if (g->ev_used >= 4096) prof_drain(g);
    if (2 * (size_t)g->ev_used + 1 >= g->ev_pool.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            cudaGetLastError();
            *ev = -1;
            return;
        }
        g->ev_pool.push_back(a);
        g->ev_pool.push_back(b);
    }
    *ev = g->ev_used++;
    cudaEventRecord(g->ev_pool[2 * *ev], g->stream);
}

void prof_end(cg_grids* g, int slot, int ev) {
    if (ev < 0) return;
    cudaEventRecord(g->ev_pool[2 * ev + 1], g->stream);
    g->pending.push_back({slot, ev});
}

// ---------------------------------------------------------------------------
// Buffers that grow with the particle count
// ---------------------------------------------------------------------------
cg_status ensure_partials(cg_grids* g, long long n) {
    const long long bulk_blk = (g->gd.nbulk + 7) / 8;   // cell kernels run 8 cells (warps) per block
    const long long fine_blk = (g->gd.nfine + 255) / 256;
    (void)n;
    const long long proj_blk = (g->gd.r == 2 || g->gd.r == 4 || g->gd.r == 8) ? bulk_blk : fine_blk;
    const long long part_blk = std::max(bulk_blk, (long long)g->num_sms * 8);
    const long long need = part_blk * (1 + kDragCellSums) + proj_blk * 6;
    if (need > g->part_cap) {
        dfree(g->partials);
        g->part_cap = 0;
        CG_TRY(dalloc(&g->partials, 2 * g->tsize * need));
        g->part_cap = need;
    }
    g->part_off[PS_VOL] = 0;
    g->part_off[PS_PROJ] = part_blk;
    g->part_off[PS_DRAG] = part_blk + proj_blk * 6;
    return CG_OK;
}

cg_status ensure_particle_capacity(cg_grids* g, long long n) {
    CG_TRY(ensure_partials(g, n));
    if (n <= g->cap) return CG_OK;
    const long long cap = ((n + kSortTile - 1) / kSortTile) * kSortTile;
    dfree(g->key);
    dfree(g->key1);
    dfree(g->val1);
    dfree(g->key2);
    dfree(g->val2);
    dfree(g->perm);
    dfree(g->key_sorted);
    dfree(g->inv_perm);
    dfree(g->vol);
    dfree(g->vol_sorted);
    dfree(g->Fs);
    dfree(g->hist);
    dfree(g->scan_part);
    dfree(g->rb_rid);
    dfree(g->rb_rkn);
    dfree(g->rb_mov);
    dfree(g->rb_arr);
    dfree(g->rb_small);
    g->cap = -1;
    g->n_binned = -1;
    g->hint_n = -1;
    g->hint_ident = nullptr;
    CG_TRY(dalloc(&g->key, sizeof(int32_t) * cap));
    CG_TRY(dalloc(&g->key1, sizeof(int32_t) * cap));
    CG_TRY(dalloc(&g->val1, sizeof(int32_t) * cap));
    CG_TRY(dalloc(&g->key2, sizeof(int32_t) * cap));
    CG_TRY(dalloc(&g->val2, sizeof(int32_t) * cap));
    CG_TRY(dalloc(&g->perm, sizeof(int32_t) * cap));
    CG_TRY(dalloc(&g->key_sorted, sizeof(int32_t) * cap));
    CG_TRY(dalloc(&g->inv_perm, sizeof(int32_t) * cap));
    CG_TRY(dalloc(&g->vol, g->tsize * cap));
    CG_TRY(dalloc(&g->vol_sorted, g->tsize * cap));
    CG_TRY(dalloc(&g->Fs, 4 * g->tsize * cap));
    const long long ntiles = cap / kSortTile;
    const int maxbits = std::max(g->pass_bits[0], std::max(g->pass_bits[1], g->pass_bits[2]));
    // digit histograms of the digit sort, or the large-cell list of the
    // default sort (at most cap / 257 cells after a count)
    g->hist_cap = std::max<long long>(ntiles << maxbits, cap / 256 + 2);
    CG_TRY(dalloc(&g->hist, sizeof(int32_t) * g->hist_cap));
    // incremental rebinning: records per old slot, room for every particle to
    // move (each block of old slots has its own part of the mover list), the
    // arrival lists, per-cell and per-block counts
    g->rb_nblk = (cap + kRebinTile - 1) / kRebinTile;
    CG_TRY(dalloc(&g->rb_rid, sizeof(int32_t) * cap));
    CG_TRY(dalloc(&g->rb_rkn, sizeof(int32_t) * cap));
    CG_TRY(dalloc(&g->rb_mov, sizeof(int2) * g->rb_nblk * kRebinTile));
    CG_TRY(dalloc(&g->rb_arr, sizeof(int2) * cap));
    CG_TRY(dalloc(&g->rb_small, sizeof(int32_t) * rebin_small_ints(g->gd.nbulk, g->rb_nblk)));
    const long long cells_blk = (g->gd.nbulk + 1 + kScanItems - 1) / kScanItems;
    g->scan_cap = std::max((g->hist_cap + kScanItems - 1) / kScanItems + cells_blk,
                           2 * cells_blk + (g->rb_nblk + 1 + kScanItems - 1) / kScanItems);
    CG_TRY(dalloc(&g->scan_part, sizeof(int32_t) * g->scan_cap));
    g->cap = cap;
    return CG_OK;
}

}  // namespace cg

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* cg_status_string(cg_status s) {
    switch (s) {
        case CG_OK: return "ok";
        case CG_ERR_INVALID_ARG: return "invalid argument";
        case CG_ERR_CUDA: return "CUDA runtime error";
        case CG_ERR_OOM: return "device out of memory";
        case CG_ERR_NOT_BINNED: return "particles not binned for this count";
        case CG_ERR_OUT_OF_RANGE: return "size beyond a documented limit";
        case CG_ERR_TIMEOUT: return "bounded device wait gave up";
        case CG_ERR_NONFINITE: return "non-finite input";
    }
    return "unknown status";
}

static void free_all(cg_grids* g) {
    dfree(g->key);
    dfree(g->key1);
    dfree(g->val1);
    dfree(g->key2);
    dfree(g->val2);
    dfree(g->perm);
    dfree(g->key_sorted);
    dfree(g->inv_perm);
    dfree(g->vol);
    dfree(g->vol_sorted);
    dfree(g->Fs);
    dfree(g->hist);
    dfree(g->scan_part);
    dfree(g->rb_rid);
    dfree(g->rb_rkn);
    dfree(g->rb_mov);
    dfree(g->rb_arr);
    dfree(g->rb_small);
    dfree(g->cell_start);
    dfree(g->bulk4);
    dfree(g->eps_t);
    dfree(g->partials);
    dfree(g->sums_scratch);
    dfree(g->status);
    for (HostStage& S : g->hs) {
        DevBuf* st[] = {&S.pos, &S.vel, &S.ufine, &S.eps, &S.ub, &S.var, &S.Sb,
                        &S.F,   &S.Sf,  &S.epsf,  &S.sums, &S.cell, &S.perm, &S.cs};
        for (DevBuf* b : st) {
            dfree(b->p);
            b->bytes = 0;
        }
        cudaEvent_t evs[] = {S.in_done, S.comp_done, S.out_done};
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
        S.in_done = S.comp_done = S.out_done = nullptr;
        S.used = false;
    }
    dfree(g->fresh4.p);
    g->fresh4.bytes = 0;
    if (g->part_out) cudaEventDestroy(g->part_out);
    g->part_out = nullptr;
    g->part_pos = g->part_vel = nullptr;
    if (g->h2d) cudaStreamDestroy(g->h2d);
    if (g->d2h) cudaStreamDestroy(g->d2h);
    g->h2d = g->d2h = nullptr;
    for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
    g->ev_pool.clear();
    cudaEvent_t evs[] = {g->ev_fork, g->ev_avg, g->ev_pack, g->ev_epsf};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (g->aux) cudaStreamDestroy(g->aux);
    g->aux = nullptr;
}

cg_status cg_create_grids(const cg_grid_desc* desc, void* cuda_stream, cg_grids** out) {
    if (!out) return CG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!desc) return CG_ERR_INVALID_ARG;
    const cg_grid_desc& d = *desc;
    if (!finite3(d.origin) || !finite3(d.extent) || !finite3(d.gravity)) return CG_ERR_INVALID_ARG;
    if (d.ratio < 1) return CG_ERR_INVALID_ARG;
    long long nbulk = 1, nfine = 1;
    int nb[3];
    for (int a = 0; a < 3; ++a) {
        if (!(d.extent[a] > 0.0) || d.fine_n[a] < 1 || d.fine_n[a] % d.ratio != 0) return CG_ERR_INVALID_ARG;
        nb[a] = d.fine_n[a] / d.ratio;
        if (nb[a] < 2) return CG_ERR_INVALID_ARG;
        // the fine count is at most 2^31 - 1, so each factor is too and the
        // running products (checked as they grow) cannot overflow 64 bits
        nbulk *= nb[a];
        nfine *= d.fine_n[a];
        if (nbulk > (1LL << kMaxBulkBits) || nfine > 2147483647LL) return CG_ERR_OUT_OF_RANGE;
    }
    if (d.prec != CG_FP32 && d.prec != CG_FP64) return CG_ERR_INVALID_ARG;
    if (d.law != CG_DRAG_DI_FELICE && d.law != CG_DRAG_ERGUN_WEN_YU) return CG_ERR_INVALID_ARG;
    if (d.interp != CG_INTERP_TRILINEAR && d.interp != CG_INTERP_CELL) return CG_ERR_INVALID_ARG;
    if (!sort_choice_valid(d.sort_digits)) return CG_ERR_INVALID_ARG;
    if (d.stencil != CG_STENCIL_GATHER && d.stencil != CG_STENCIL_WINDOW) return CG_ERR_INVALID_ARG;
    if (!(d.rho_f > 0.0) || !(d.mu_f > 0.0) || !(d.rho_p > 0.0) || !isfinite(d.rho_f) || !isfinite(d.mu_f) ||
        !isfinite(d.rho_p))
        return CG_ERR_INVALID_ARG;
    if (!(d.eps_switch > 0.0 && d.eps_switch <= 1.0)) return CG_ERR_INVALID_ARG;
    if (!(d.eps_min >= 0.0 && d.eps_min < 1.0)) return CG_ERR_INVALID_ARG;
    if (nbulk > (1LL << kMaxBulkBits) || nfine > 2147483647LL) return CG_ERR_OUT_OF_RANGE;

    cg_grids* g = new (std::nothrow) cg_grids();
    if (!g) return CG_ERR_OOM;
    g->desc = d;
    g->fp64 = d.prec == CG_FP64;
    g->tsize = g->fp64 ? 8 : 4;
    g->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return CG_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);

    GridDev& gd = g->gd;
    memset(&gd, 0, sizeof gd);
    gd.r = d.ratio;
    gd.nbulk = nbulk;
    gd.nfine = nfine;
    double h[3];
    for (int a = 0; a < 3; ++a) {
        gd.nb[a] = nb[a];
        gd.nf[a] = d.fine_n[a];
        gd.x0[a] = d.origin[a];
        gd.xhi[a] = d.origin[a] + d.extent[a];
        gd.H[a] = d.extent[a] / (double)nb[a];
        h[a] = d.extent[a] / (double)d.fine_n[a];
        gd.invH[a] = 1.0 / gd.H[a];
        gd.x0f[a] = (float)d.origin[a];
        gd.xhif[a] = (float)gd.xhi[a];
        gd.invHf[a] = (float)gd.invH[a];
        gd.ax0f[a] = (float)fabs(d.origin[a] * gd.invH[a]);
        split_ff(d.origin[a], gd.x0h[a], gd.x0l[a]);
        split_ff(gd.invH[a], gd.ihh[a], gd.ihl[a]);
        split_ff(-(d.origin[a] / gd.H[a] + 0.5), gd.xbh[a], gd.xbl[a]);
    }
    gd.VB = gd.H[0] * gd.H[1] * gd.H[2];
    gd.invVB = 1.0 / gd.VB;
    gd.Vf = h[0] * h[1] * h[2];
    gd.invVBf = (float)gd.invVB;
    gd.VBf = (float)gd.VB;
    gd.Vff = (float)gd.Vf;
    split_ff(gd.VB, gd.VBh, gd.VBl);
    split_ff(gd.Vf, gd.Vfh, gd.Vfl);
    split_ff(gd.invVB, gd.ivBh, gd.ivBl);
    gd.law = d.law;
    gd.interp = d.interp;
    gd.rho_f = d.rho_f;
    gd.mu_f = d.mu_f;
    gd.rho_p = d.rho_p;
    gd.eps_switch = d.eps_switch;
    gd.eps_min = d.eps_min;
    for (int a = 0; a < 3; ++a) gd.g[a] = d.gravity[a];

    g->bulk_bits = std::max(1, ceil_log2(nbulk));
    g->npasses = split_passes(g->bulk_bits, g->pass_bits, d.sort_digits >= 6 ? d.sort_digits : 0);

    cg_status st = CG_OK;
    if (st == CG_OK) st = dalloc(&g->cell_start, sizeof(int32_t) * (nbulk + 1));
    if (st == CG_OK) st = dalloc(&g->bulk4, 4 * g->tsize * nbulk);
    if (st == CG_OK) st = dalloc(&g->eps_t, g->tsize * nbulk);
    if (st == CG_OK) st = dalloc(&g->sums_scratch, sizeof(double) * CG_NSUMS);
    if (st == CG_OK) st = dalloc(&g->status, sizeof(unsigned long long) * kNumSlots);
    if (st == CG_OK && cudaMemset(g->status, 0, sizeof(unsigned long long) * kNumSlots) != cudaSuccess)
        st = CG_ERR_CUDA;
    if (st == CG_OK && cudaStreamCreateWithFlags(&g->aux, cudaStreamNonBlocking) != cudaSuccess) st = CG_ERR_CUDA;
    cudaEvent_t* evs[] = {&g->ev_fork, &g->ev_avg, &g->ev_pack, &g->ev_epsf};
    for (cudaEvent_t* e : evs)
        if (st == CG_OK && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) st = CG_ERR_CUDA;
    if (st == CG_OK) st = ensure_particle_capacity(g, 1);
    if (st != CG_OK) {
        free_all(g);
        delete g;
        return st;
    }
    *out = g;
    return CG_OK;
}

cg_status cg_debug_fail_alloc_after(int64_t k) {
    if (k < -1) return CG_ERR_INVALID_ARG;
    g_alloc_fail_after.store(k);
    return CG_OK;
}

cg_status cg_destroy_grids(cg_grids* g) {
    if (!g) return CG_OK;
    cudaStreamSynchronize(g->stream);
    cudaGetLastError();
    free_all(g);
    delete g;
    return CG_OK;
}

cg_status cg_set_stream(cg_grids* g, void* cuda_stream) {
    CG_TRY(check_handle(g));
    g->stream = (cudaStream_t)cuda_stream;
    return CG_OK;
}

cg_status cg_grid_dims(const cg_grids* g, int32_t bulk_n[3], int64_t* n_bulk, int64_t* n_fine) {
    CG_TRY(check_handle(g));
    if (bulk_n)
        for (int a = 0; a < 3; ++a) bulk_n[a] = g->gd.nb[a];
    if (n_bulk) *n_bulk = g->gd.nbulk;
    if (n_fine) *n_fine = g->gd.nfine;
    return CG_OK;
}

static cg_status check_n(long long n) { return (n < 0 || n > 2147483647LL) ? CG_ERR_OUT_OF_RANGE : CG_OK; }

static cg_status copy_bins(cg_grids* g, long long n, int32_t* cell_out, int32_t* perm_out, int32_t* cs_out) {
    if (cell_out && n) CG_TRY(ensure_keys(g, n));
    if (cell_out && n)
        CG_CUDA(cudaMemcpyAsync(cell_out, g->key, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, g->stream));
    if (perm_out && n)
        CG_CUDA(cudaMemcpyAsync(perm_out, g->perm, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, g->stream));
    if (cs_out)
        CG_CUDA(cudaMemcpyAsync(cs_out, g->cell_start, sizeof(int32_t) * (g->gd.nbulk + 1),
                                cudaMemcpyDeviceToDevice, g->stream));
    return CG_OK;
}

cg_status cg_bin_particles(cg_grids* g, int64_t n, const void* pos_d, int32_t* cell_out, int32_t* perm_out,
                           int32_t* cell_start_out) {
    CG_TRY(check_handle(g));
    CG_TRY(check_n(n));
    if (n > 0 && (!pos_d || !aligned16(pos_d))) return CG_ERR_INVALID_ARG;
    CG_TRY(ensure_particle_capacity(g, n));
    CG_TRY(launch_bin(g, n, pos_d));
    return copy_bins(g, n, cell_out, perm_out, cell_start_out);
}

cg_status cg_reorder_particles(cg_grids* g, int64_t n, const void* pos_d, const void* vel, void* pos_out,
                               void* vel_out) {
    CG_TRY(check_handle(g));
    CG_TRY(check_n(n));
    if ((vel == nullptr) != (vel_out == nullptr)) return CG_ERR_INVALID_ARG;
    if (n == 0) return CG_OK;
    if (!pos_d || !pos_out || !aligned16(pos_d) || !aligned16(pos_out)) return CG_ERR_INVALID_ARG;
    if (vel && (!aligned16(vel) || !aligned16(vel_out))) return CG_ERR_INVALID_ARG;
    const size_t bytes = 4 * g->tsize * (size_t)n;
    auto overlap = [&](const void* a, const void* b) {
        const char *x = (const char*)a, *y = (const char*)b;
        return x < y + bytes && y < x + bytes;
    };
    if (overlap(pos_d, pos_out) || (vel && (overlap(vel, vel_out) || overlap(pos_d, vel_out) || overlap(vel, pos_out))))
        return CG_ERR_INVALID_ARG;
    if (g->n_binned != n) return CG_ERR_NOT_BINNED;
    return launch_reorder(g, n, pos_d, vel, pos_out, vel_out);
}

cg_status cg_deposit(cg_grids* g, int32_t kind, int64_t n, const void* per_particle, void* bulk_out) {
    CG_TRY(check_handle(g));
    CG_TRY(check_n(n));
    if (kind != CG_DEP_VOLUME && kind != CG_DEP_MOMENTUM) return CG_ERR_INVALID_ARG;
    if (!bulk_out || (n > 0 && !per_particle)) return CG_ERR_INVALID_ARG;
    if (kind == CG_DEP_VOLUME && n > 0 && !aligned16(per_particle)) return CG_ERR_INVALID_ARG;
    if (g->n_binned != n) return CG_ERR_NOT_BINNED;
    if (kind == CG_DEP_VOLUME) return launch_deposit_volume(g, n, per_particle, (double*)bulk_out, false);
    return launch_deposit_momentum(g, n, per_particle, bulk_out);
}

cg_status cg_average_fine_to_bulk(cg_grids* g, const void* u_fine, void* u_bulk, void* var_bulk) {
    CG_TRY(check_handle(g));
    if (!u_fine || !u_bulk || !aligned16(u_fine)) return CG_ERR_INVALID_ARG;
    return launch_average(g, u_fine, u_bulk, var_bulk);
}

cg_status cg_drag(cg_grids* g, int64_t n, const void* pos_d, const void* vel, const double* eps_bulk,
                  const void* u_bulk, void* force_out, void* S_bulk_out, const cg_mlp* mlp) {
    CG_TRY(check_handle(g));
    CG_TRY(check_n(n));
    if (!eps_bulk || !u_bulk) return CG_ERR_INVALID_ARG;
    if (n > 0 && (!pos_d || !vel || !force_out || !aligned16(pos_d) || !aligned16(vel))) return CG_ERR_INVALID_ARG;
    if (S_bulk_out && g->n_binned != n) return CG_ERR_NOT_BINNED;
    const void* var_stale = nullptr;
    const void* u_fine = nullptr;
    int32_t age = 1;
    if (mlp) {
        if (g->fp64) return CG_ERR_INVALID_ARG;
        CG_TRY(mlp_bound_inputs(mlp, &var_stale, &u_fine, &age));
    }
    CG_TRY(ensure_particle_capacity(g, n));
    CG_TRY(launch_pack(g, eps_bulk, u_bulk, false));
    if (mlp)
        return launch_drag_learned(g, mlp, n, const_cast<void*>(pos_d), const_cast<void*>(vel), var_stale, u_fine,
                                   age, force_out, S_bulk_out, 0.0);
    return launch_drag(g, n, pos_d, vel, force_out, S_bulk_out, false, 0.0);
}

cg_status cg_project_bulk_to_fine(cg_grids* g, int32_t ncomp, const void* bulk, void* fine_out) {
    CG_TRY(check_handle(g));
    if (ncomp < 1 || ncomp > 4 || !bulk || !fine_out || !aligned16(fine_out)) return CG_ERR_INVALID_ARG;
    const void* in[4] = {nullptr, nullptr, nullptr, nullptr};
    void* out[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int c = 0; c < ncomp; ++c) {
        in[c] = (const char*)bulk + (size_t)c * g->gd.nbulk * g->tsize;
        out[c] = (char*)fine_out + (size_t)c * g->gd.nfine * g->tsize;
    }
    return launch_project(g, ncomp, in, out, false);
}

// Launch f on the auxiliary stream (the handle's launch macros use g->stream).
// While per-kernel timing is on, everything stays on the main stream so that
// each kernel's event pair measures that kernel alone.
extern "C++" {
template <typename Fn>
static cg_status on_aux(cg_grids* g, Fn f) {
    if (g->prof) return f();
    cudaStream_t main = g->stream;
    g->stream = g->aux;
    cg_status s = f();
    g->stream = main;
    return s;
}
}

// One coupling step.  Fork / join on the auxiliary stream:
//   main: bin -> porosity --(avg)--> drag -> reaction -> project S --(eps_f)--> sums
//   aux :  average fine -> bulk  \-(porosity)-> project eps
// The averaging reads only the fine field and the porosity projection only
// the packed porosity, so both overlap the latency-bound particle kernels.
//
// With a learned closure and no refresh the averaging is skipped: u_bulk and
// var_bulk are inputs (the record of the last refresh) and the drag is the
// learned kernel, which reads the fine field only for its fallback rows.
// sorted_out (nullable): the particles leave in this binning's order in
// these arrays (cg_step_sorted), and the next binning of them starts from it.
static cg_status step_impl(cg_grids* g, const cg_particles* p, const void* u_fine, const cg_step_out* o,
                           double dt, const cg_mlp* mlp = nullptr, int32_t age = 0,
                           const cg_particles* sorted_out = nullptr) {
    const long long n = p->n;
    CG_TRY(ensure_particle_capacity(g, n));
    if (o->implicit_bulk && mlp) return CG_ERR_INVALID_ARG;   // no drag factor in the learned form
    if (o->implicit_bulk && n > 0) CG_TRY(grow_buf(g->Bs, 4 * g->tsize * (size_t)g->cap));
    for (int r = 0; r < PS_NREG; ++r) g->part_blocks[r] = -1;
    cudaStream_t side = g->prof ? g->stream : g->aux;
    CG_CUDA(cudaEventRecord(g->ev_fork, g->stream));
    CG_CUDA(cudaStreamWaitEvent(side, g->ev_fork, 0));
    // the drag's packed record (eps, u) is written by the kernels that form its
    // parts: the average (u, on the side stream), the binning (eps = 1 in every
    // cell) and the porosity deposit (eps of occupied cells); with a closure
    // or no particles it is packed from the outputs instead
    const bool fused = !mlp && n > 0;
    void* eps_t = o->eps_fine ? g->eps_t : nullptr;
    if (!mlp)
        CG_TRY(on_aux(g, [&] { return launch_average(g, u_fine, o->u_bulk, o->var_bulk, fused ? g->bulk4 : nullptr); }));
    CG_CUDA(cudaEventRecord(g->ev_avg, side));
    if (fused) CG_TRY(launch_bin(g, n, p->pos_d, o->eps_bulk, g->bulk4, eps_t));
    else CG_TRY(launch_bin(g, n, p->pos_d, o->eps_bulk));
    CG_TRY(copy_bins(g, n, o->cell, o->perm, o->cell_start));
    // sorted diameters of this binning
    if (fused) CG_TRY(launch_deposit_volume(g, n, nullptr, o->eps_bulk, true, true, g->bulk4, eps_t));
    else CG_TRY(launch_deposit_volume(g, n, nullptr, o->eps_bulk, true, true));
    if (!fused) {
        CG_CUDA(cudaStreamWaitEvent(g->stream, g->ev_avg, 0));
        CG_TRY(launch_pack(g, o->eps_bulk, o->u_bulk, o->eps_fine != nullptr));
    }
    if (o->eps_fine) {
        CG_CUDA(cudaEventRecord(g->ev_pack, g->stream));
        CG_CUDA(cudaStreamWaitEvent(side, g->ev_pack, 0));
        const void* ein[4] = {g->eps_t, nullptr, nullptr, nullptr};
        void* eout[4] = {o->eps_fine, nullptr, nullptr, nullptr};
        CG_TRY(on_aux(g, [&] { return launch_project(g, 1, ein, eout, false); }));
    }
    if (fused) CG_CUDA(cudaStreamWaitEvent(g->stream, g->ev_avg, 0));
    CG_CUDA(cudaEventRecord(g->ev_epsf, side));
    if (mlp)
        CG_TRY(launch_drag_learned(g, mlp, n, p->pos_d, p->vel, o->var_bulk, u_fine, age, o->force, o->S_bulk,
                                   dt));
    else
        CG_TRY(launch_drag(g, n, p->pos_d, p->vel, o->force, o->S_bulk, true, dt, o->implicit_bulk,
                           sorted_out ? sorted_out->pos_d : nullptr, sorted_out ? sorted_out->vel : nullptr));
    // the binning above lists the sorted output's particle i at slot i
    if (sorted_out && g->n_binned == n) g->hint_ident = sorted_out->pos_d;
    const size_t bs = (size_t)g->gd.nbulk * g->tsize, fs = (size_t)g->gd.nfine * g->tsize;
    const void* in[4] = {o->S_bulk, (const char*)o->S_bulk + bs, (const char*)o->S_bulk + 2 * bs, nullptr};
    void* out[4] = {o->S_fine, (char*)o->S_fine + fs, (char*)o->S_fine + 2 * fs, nullptr};
    CG_TRY(launch_project(g, 3, in, out, true));
    if (o->implicit_fine) {
        const void* ci[4];
        void* co[4];
        for (int c = 0; c < 4; ++c) {
            ci[c] = (const char*)o->implicit_bulk + c * bs;
            co[c] = (char*)o->implicit_fine + c * fs;
        }
        CG_TRY(launch_project(g, 4, ci, co, false));
    }
    CG_CUDA(cudaStreamWaitEvent(g->stream, g->ev_epsf, 0));
    CG_TRY(launch_sums(g, o->sums ? o->sums : g->sums_scratch));
    return CG_OK;
}

static cg_status check_step_args(const cg_particles* p, const void* u_fine, const cg_step_out* o, double dt,
                                 bool device) {
    if (!p || !o || !u_fine) return CG_ERR_INVALID_ARG;
    CG_TRY(check_n(p->n));
    if (!(dt >= 0.0) || !isfinite(dt)) return CG_ERR_INVALID_ARG;
    if (p->n > 0 && (!p->pos_d || !p->vel || !o->force)) return CG_ERR_INVALID_ARG;
    if (!o->eps_bulk || !o->u_bulk || !o->S_bulk || !o->S_fine) return CG_ERR_INVALID_ARG;
    if (o->implicit_fine && !o->implicit_bulk) return CG_ERR_INVALID_ARG;
    if (!device && (o->implicit_bulk || o->implicit_fine)) return CG_ERR_INVALID_ARG;   // device entries only
    if (device) {
        if (p->n > 0 && (!aligned16(p->pos_d) || !aligned16(p->vel))) return CG_ERR_INVALID_ARG;
        if (!aligned16(u_fine) || !aligned16(o->S_fine) || (o->eps_fine && !aligned16(o->eps_fine)))
            return CG_ERR_INVALID_ARG;
    }
    return CG_OK;
}

cg_status cg_step(cg_grids* g, const cg_particles* p, const void* u_fine, const cg_step_out* out, double dt) {
    CG_TRY(check_handle(g));
    CG_TRY(check_step_args(p, u_fine, out, dt, true));
    return step_impl(g, p, u_fine, out, dt);
}

cg_status cg_step_sorted(cg_grids* g, const cg_particles* p, const cg_particles* p_out, const void* u_fine,
                         const cg_step_out* out, double dt) {
    CG_TRY(check_handle(g));
    CG_TRY(check_step_args(p, u_fine, out, dt, true));
    if (!p_out || p_out->n != p->n) return CG_ERR_INVALID_ARG;
    const long long n = p->n;
    if (n > 0) {
        if (!p_out->pos_d || !p_out->vel || !aligned16(p_out->pos_d) || !aligned16(p_out->vel))
            return CG_ERR_INVALID_ARG;
        const size_t bytes = 4 * g->tsize * (size_t)n;
        auto overlap = [&](const void* a, const void* b) {
            const char *x = (const char*)a, *y = (const char*)b;
            return x < y + bytes && y < x + bytes;
        };
        const void* ins[2] = {p->pos_d, p->vel};
        const void* outs[2] = {p_out->pos_d, p_out->vel};
        if (overlap(outs[0], outs[1])) return CG_ERR_INVALID_ARG;
        for (const void* a : outs)
            for (const void* b : ins)
                if (overlap(a, b)) return CG_ERR_INVALID_ARG;
    }
    return step_impl(g, p, u_fine, out, dt, nullptr, 0, p_out);
}

cg_status cg_step_learned(cg_grids* g, const cg_particles* p, const void* u_fine, const cg_step_out* out, double dt,
                          const cg_mlp* mlp, int32_t age) {
    CG_TRY(check_handle(g));
    CG_TRY(check_step_args(p, u_fine, out, dt, true));
    if (!mlp || g->fp64 || !out->var_bulk || age < 0) return CG_ERR_INVALID_ARG;
    if (out->implicit_bulk || out->implicit_fine) return CG_ERR_INVALID_ARG;   // no drag factor in the learned form
    return step_impl(g, p, u_fine, out, dt, age == 0 ? nullptr : mlp, age);
}

// Host-buffer steps.  Each call takes the next of two staging sets: its
// inputs go in on the h2d stream (after the set's previous outputs have
// left), the step runs on the handle's stream, and the outputs go out on the
// d2h stream; so the copies of consecutive steps overlap each other and the
// compute (one direction each way at a time).  A step that advances its
// particles (dt > 0) sends them back first; a later call whose particle
// arrays are those host arrays copies them in only after they have arrived
// (its fluid field goes in meanwhile), so advancing steps may be enqueued
// back to back on the same arrays.
static cg_status step_host_enqueue(cg_grids* g, const cg_particles* p, const void* u_fine, const cg_step_out* out,
                                   double dt) {
    const long long n = p->n;
    const size_t ts = g->tsize, nb = (size_t)g->gd.nbulk, nf = (size_t)g->gd.nfine;
    const size_t pbytes = 4 * ts * (size_t)std::max(1LL, n);
    HostStage& S = g->hs[g->hs_next];
    if (!g->h2d) {
        CG_CUDA(cudaStreamCreateWithFlags(&g->h2d, cudaStreamNonBlocking));
        CG_CUDA(cudaStreamCreateWithFlags(&g->d2h, cudaStreamNonBlocking));
    }
    if (!S.in_done) {
        CG_CUDA(cudaEventCreateWithFlags(&S.in_done, cudaEventDisableTiming));
        CG_CUDA(cudaEventCreateWithFlags(&S.comp_done, cudaEventDisableTiming));
        CG_CUDA(cudaEventCreateWithFlags(&S.out_done, cudaEventDisableTiming));
    }
    // the set's buffers may only be regrown once nothing uses them
    if (S.used) CG_CUDA(cudaEventSynchronize(S.out_done));
    CG_TRY(ensure_buf(S.pos, pbytes));
    CG_TRY(ensure_buf(S.vel, pbytes));
    CG_TRY(ensure_buf(S.ufine, 3 * ts * nf));
    CG_TRY(ensure_buf(S.eps, sizeof(double) * nb));
    CG_TRY(ensure_buf(S.ub, 3 * ts * nb));
    CG_TRY(ensure_buf(S.Sb, 3 * ts * nb));
    CG_TRY(ensure_buf(S.F, 3 * ts * (size_t)std::max(1LL, n)));
    CG_TRY(ensure_buf(S.Sf, 3 * ts * nf));
    if (out->var_bulk) CG_TRY(ensure_buf(S.var, ts * nb));
    if (out->eps_fine) CG_TRY(ensure_buf(S.epsf, ts * nf));
    if (out->sums) CG_TRY(ensure_buf(S.sums, sizeof(double) * CG_NSUMS));
    if (out->cell) CG_TRY(ensure_buf(S.cell, sizeof(int32_t) * (size_t)std::max(1LL, n)));
    if (out->perm) CG_TRY(ensure_buf(S.perm, sizeof(int32_t) * (size_t)std::max(1LL, n)));
    if (out->cell_start) CG_TRY(ensure_buf(S.cs, sizeof(int32_t) * (nb + 1)));
    // the particle scratch too, so that a failed allocation enqueues nothing
    CG_TRY(ensure_particle_capacity(g, n));
    g->hs_next ^= 1;

    // inputs in: the fluid field, then the particles (once a step that
    // advanced these host arrays has sent them back)
    if (S.used) CG_CUDA(cudaStreamWaitEvent(g->h2d, S.out_done, 0));
    CG_CUDA(cudaMemcpyAsync(S.ufine.p, u_fine, 3 * ts * nf, cudaMemcpyHostToDevice, g->h2d));
    if (n > 0) {
        if (g->part_out && (p->pos_d == g->part_pos || p->vel == g->part_vel))
            CG_CUDA(cudaStreamWaitEvent(g->h2d, g->part_out, 0));
        CG_CUDA(cudaMemcpyAsync(S.pos.p, p->pos_d, 4 * ts * n, cudaMemcpyHostToDevice, g->h2d));
        CG_CUDA(cudaMemcpyAsync(S.vel.p, p->vel, 4 * ts * n, cudaMemcpyHostToDevice, g->h2d));
    }
    CG_CUDA(cudaEventRecord(S.in_done, g->h2d));
    S.used = true;

    // the step
    CG_CUDA(cudaStreamWaitEvent(g->stream, S.in_done, 0));
    cg_particles dp = {n, S.pos.p, S.vel.p};
    cg_step_out d = {};   // every field the host call does not map stays null
    d.eps_bulk = (double*)S.eps.p;
    d.u_bulk = S.ub.p;
    d.var_bulk = out->var_bulk ? S.var.p : nullptr;
    d.S_bulk = S.Sb.p;
    d.force = S.F.p;
    d.S_fine = S.Sf.p;
    d.eps_fine = out->eps_fine ? S.epsf.p : nullptr;
    d.sums = out->sums ? (double*)S.sums.p : nullptr;
    d.cell = out->cell ? (int32_t*)S.cell.p : nullptr;
    d.perm = out->perm ? (int32_t*)S.perm.p : nullptr;
    d.cell_start = out->cell_start ? (int32_t*)S.cs.p : nullptr;
    CG_TRY(step_impl(g, &dp, S.ufine.p, &d, dt));
    CG_CUDA(cudaEventRecord(S.comp_done, g->stream));

    // outputs out
    cudaStream_t s = g->d2h;
    CG_CUDA(cudaStreamWaitEvent(s, S.comp_done, 0));
    auto d2h = [&](void* dst, const void* src, size_t bytes) -> cg_status {
        if (dst && bytes) CG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
        return CG_OK;
    };
    if (dt > 0.0 && n > 0) {
        // the advanced particles first: the next step on these arrays waits for them
        if (!g->part_out) CG_CUDA(cudaEventCreateWithFlags(&g->part_out, cudaEventDisableTiming));
        CG_TRY(d2h(p->pos_d, S.pos.p, 4 * ts * n));
        CG_TRY(d2h(p->vel, S.vel.p, 4 * ts * n));
        CG_CUDA(cudaEventRecord(g->part_out, s));
        g->part_pos = p->pos_d;
        g->part_vel = p->vel;
    }
    CG_TRY(d2h(out->eps_bulk, d.eps_bulk, sizeof(double) * nb));
    CG_TRY(d2h(out->u_bulk, d.u_bulk, 3 * ts * nb));
    CG_TRY(d2h(out->var_bulk, d.var_bulk, ts * nb));
    CG_TRY(d2h(out->S_bulk, d.S_bulk, 3 * ts * nb));
    CG_TRY(d2h(out->force, d.force, 3 * ts * n));
    CG_TRY(d2h(out->S_fine, d.S_fine, 3 * ts * nf));
    CG_TRY(d2h(out->eps_fine, d.eps_fine, ts * nf));
    CG_TRY(d2h(out->sums, d.sums, sizeof(double) * CG_NSUMS));
    CG_TRY(d2h(out->cell, d.cell, sizeof(int32_t) * n));
    CG_TRY(d2h(out->perm, d.perm, sizeof(int32_t) * n));
    CG_TRY(d2h(out->cell_start, d.cell_start, sizeof(int32_t) * (nb + 1)));
    CG_CUDA(cudaEventRecord(S.out_done, s));
    return CG_OK;
}

static cg_status step_host_wait(cg_grids* g) {
    if (g->d2h && cudaStreamSynchronize(g->d2h) != cudaSuccess) return CG_ERR_CUDA;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return CG_ERR_CUDA;
    return CG_OK;
}

cg_status cg_step_host(cg_grids* g, const cg_particles* p, const void* u_fine, const cg_step_out* out,
                       double dt) {
    CG_TRY(check_handle(g));
    CG_TRY(check_step_args(p, u_fine, out, dt, false));
    CG_TRY(step_host_enqueue(g, p, u_fine, out, dt));
    return step_host_wait(g);
}

cg_status cg_step_host_async(cg_grids* g, const cg_particles* p, const void* u_fine, const cg_step_out* out,
                             double dt) {
    CG_TRY(check_handle(g));
    CG_TRY(check_step_args(p, u_fine, out, dt, false));
    return step_host_enqueue(g, p, u_fine, out, dt);
}

cg_status cg_step_host_wait(cg_grids* g) {
    CG_TRY(check_handle(g));
    return step_host_wait(g);
}

cg_status cg_sync_status(cg_grids* g, uint32_t* flags, int64_t* counts) {
    CG_TRY(check_handle(g));
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
        cudaGetLastError();
        return CG_ERR_CUDA;
    }
    unsigned long long h[kNumSlots];
    CG_CUDA(cudaMemcpy(h, g->status, sizeof h, cudaMemcpyDeviceToHost));
    CG_CUDA(cudaMemset(g->status, 0, sizeof h));
    if (flags) *flags = (uint32_t)h[ST_FLAGS];
    if (counts) {
        counts[0] = (int64_t)h[ST_OUTSIDE];
        counts[1] = (int64_t)h[ST_NONFINITE];
        counts[2] = (int64_t)h[ST_CLAMPED];
        counts[3] = (int64_t)h[ST_TIMEOUT];
        counts[4] = (int64_t)h[ST_FALLBACK];
    }
    if (h[ST_FLAGS] & CG_FLAG_TIMEOUT) return CG_ERR_TIMEOUT;
    if (h[ST_FLAGS] & CG_FLAG_NONFINITE) return CG_ERR_NONFINITE;
    return CG_OK;
}

int64_t cg_launch_count(const cg_grids* g) { return g ? g->launches : -1; }

cg_status cg_profile_enable(cg_grids* g, int32_t on) {
    CG_TRY(check_handle(g));
    if (!on) prof_drain(g);
    g->prof = on != 0;
    return CG_OK;
}

cg_status cg_profile_reset(cg_grids* g) {
    CG_TRY(check_handle(g));
    prof_drain(g);
    for (ProfSlot& s : g->slots) {
        s.launches = 0;
        s.total_ms = 0.0;
    }
    return CG_OK;
}

cg_status cg_profile_read(cg_grids* g, int32_t k, const char** name, int64_t* launches, double* total_ms,
                          int32_t* count) {
    CG_TRY(check_handle(g));
    prof_drain(g);
    if (count) *count = (int32_t)g->slots.size();
    if (k < 0 || k >= (int32_t)g->slots.size()) return name || launches || total_ms ? CG_ERR_INVALID_ARG : CG_OK;
    if (name) *name = g->slots[k].name.c_str();
    if (launches) *launches = g->slots[k].launches;
    if (total_ms) *total_ms = g->slots[k].total_ms;
    return CG_OK;
}

}  // extern "C"
