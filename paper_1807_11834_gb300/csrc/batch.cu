// batch.cu -- host runtime of the batched coupling step: many independent
// FP32 instances (uneven grids and particle counts) stepped by one
// persistent launch per phase, optionally replayed as one CUDA graph, with
// the work decomposition chosen by an autotuner.
//
// Decomposition knobs (cg_batch_config) change only how work is cut into
// blocks, never the arithmetic: the segmented sums own fixed 256-slot
// chunks of the sorted order, the sort is stable for any digit split, and
// each cell or particle is computed by one thread in a fixed order, so every
// field is bit-identical across configurations and to cg_step of the same
// instance.  Only the FP64 conservation sums, merged from per-block
// partials, may differ in their last bits.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <string>
#include <vector>

#include "batch.cuh"

using namespace cg;

struct cg_batch {
    cudaStream_t stream = nullptr;       // the batch's own stream (capturable)
    cudaStream_t user = nullptr;         // caller's stream, joined before and after a step
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int num_sms = 148;
    std::vector<cg_grids*> h;            // one handle per instance (scratch owner)
    std::vector<cg_batch_item> items;
    std::vector<BInst> hi;               // host copy of the device records
    BInst* d_inst = nullptr;
    long long* d_start = nullptr;        // [BP_COUNT][ninst + 1]
    std::vector<long long> start;        // host copy
    long long total[BP_COUNT] = {0};
    unsigned grid[BP_COUNT] = {0};
    size_t smem[BP_COUNT] = {0};
    std::vector<void*> owned;            // batch-owned device buffers
    cg_batch_config cfg;
    bool use_graph = false;
    cudaGraphExec_t gexec = nullptr;        // graph of the batched launches
    double graph_dt = -1.0;
    cudaGraphExec_t gexec_each = nullptr;   // graph of cg_step per instance
    double graph_dt_each = -1.0;
    long long launches = 0;
};

namespace {

int ceil_log2_ll(long long v) {
    int b = 0;
    while ((1LL << b) < v) ++b;
    return b;
}

long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

bool valid_config(const cg_batch_config& c) {
    return c.digit_bits >= 8 && c.digit_bits <= kMaxDigitBits && c.drag_items >= 1 && c.drag_items <= 64 &&
           c.avg_items >= 1 && c.avg_items <= 64 && c.seg_chunks >= 1 && c.seg_chunks <= 64 && c.grid_mult >= 1 &&
           c.grid_mult <= 8;
}

void free_owned(cg_batch* b) {
    for (void* p : b->owned) cudaFree(p);
    b->owned.clear();
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_start) cudaFree(b->d_start);
    b->d_inst = nullptr;
    b->d_start = nullptr;
}

cg_status dev_alloc(cg_batch* b, void** p, size_t bytes) {
    *p = nullptr;
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        return CG_ERR_OOM;
    }
    b->owned.push_back(*p);
    return CG_OK;
}

void drop_graph(cg_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->graph_dt = -1.0;
    if (b->gexec_each) cudaGraphExecDestroy(b->gexec_each);
    b->gexec_each = nullptr;
    b->graph_dt_each = -1.0;
}

// Lay out every instance's work under the configuration: pass bits,
// virtual blocks per phase, partial regions, scan jobs; allocate the
// batch-owned scratch and upload the device records.
cg_status plan(cg_batch* b) {
    const cg_batch_config& c = b->cfg;
    const int ni = (int)b->h.size();
    CG_CUDA(cudaStreamSynchronize(b->stream));   // no launch may still use the old buffers
    drop_graph(b);
    free_owned(b);
    b->hi.assign(ni, BInst());
    std::vector<long long> blocks((size_t)BP_COUNT * ni, 0);
    size_t smem_key = 0, smem_s0 = 0, smem_s1 = 0, smem_hist1 = 0;
    for (int i = 0; i < ni; ++i) {
        cg_grids* g = b->h[i];
        const cg_batch_item& it = b->items[i];
        BInst& I = b->hi[i];
        const long long n = it.particles.n, nb = g->gd.nbulk;
        I.gd = g->gd;
        I.P = phys_of<float>(g->gd);
        I.n = n;
        I.ntiles = (int)cdiv(n, kSortTile);
        // batched instances take the per-cell sort only when the descriptor
        // asks for it: over a batch of instances in random order the digit
        // sort measured faster (the per-cell sort's scattered placement and
        // per-cell work add up across instances)
        I.cellsort = g->desc.sort_digits == CG_SORT_CELLS ? 1 : 0;
        const int bits = std::max(1, ceil_log2_ll(nb));
        if (!I.cellsort && bits > 2 * c.digit_bits) return CG_ERR_OUT_OF_RANGE;
        I.npasses = I.cellsort ? 0 : bits <= c.digit_bits ? 1 : 2;
        I.b0 = I.cellsort ? 0 : I.npasses == 1 ? bits : (bits + 1) / 2;
        I.b1 = I.npasses == 2 ? bits - I.b0 : 0;
        I.pos = (float*)it.particles.pos_d;
        I.vel = (float*)it.particles.vel;
        I.u_fine = (const float*)it.u_fine;
        I.eps = it.out.eps_bulk;
        I.u_bulk = (float*)it.out.u_bulk;
        I.var = (float*)it.out.var_bulk;
        I.S_bulk = (float*)it.out.S_bulk;
        I.force = (float*)it.out.force;
        I.S_fine = (float*)it.out.S_fine;
        I.eps_fine = (float*)it.out.eps_fine;
        I.sums = it.out.sums ? it.out.sums : g->sums_scratch;
        I.key = g->key;
        I.count = g->cell_start;
        I.key1 = g->key1;
        I.val1 = g->val1;
        I.arrival = g->key2;
        I.perm = g->perm;
        I.key_sorted = g->key_sorted;
        I.inv_perm = g->inv_perm;
        I.vol = (float*)g->vol;
        I.vol_sorted = (float*)g->vol_sorted;
        I.Fs = (float*)g->Fs;
        I.bulk4 = (float*)g->bulk4;
        I.eps_t = (float*)g->eps_t;
        I.status = g->status;
        // batch-owned scratch: digit histograms, scan partials, sum partials
        const long long m0 = I.cellsort ? 0 : (long long)I.ntiles << I.b0;
        const long long m1 = (long long)I.ntiles << I.b1;
        const long long hist_m = std::max(m0, I.npasses == 2 ? m1 : 0LL);
        CG_TRY(dev_alloc(b, (void**)&I.hist, sizeof(int32_t) * hist_m));
        I.scan0.in[0] = I.count;
        I.scan0.out[0] = I.count;
        I.scan0.m[0] = nb + 1;
        I.scan0.in[1] = I.hist;
        I.scan0.out[1] = I.hist;
        I.scan0.m[1] = m0;
        I.scan0.nblk[0] = cdiv(nb + 1, kScanItems);
        I.scan0.nblk[1] = cdiv(m0, kScanItems);
        I.scan1.in[0] = I.hist;
        I.scan1.out[0] = I.hist;
        I.scan1.m[0] = I.npasses == 2 ? m1 : 0;
        I.scan1.nblk[0] = cdiv(I.scan1.m[0], kScanItems);
        I.scan1.in[1] = nullptr;
        I.scan1.out[1] = nullptr;
        I.scan1.m[1] = 0;
        I.scan1.nblk[1] = 0;
        const long long scan_blocks = std::max(I.scan0.nblk[0] + I.scan0.nblk[1], I.scan1.nblk[0]);
        CG_TRY(dev_alloc(b, (void**)&I.scan_part, sizeof(int32_t) * scan_blocks));
        // virtual blocks per phase
        long long* B = &blocks[(size_t)i];
        auto set = [&](int ph, long long v) { B[(size_t)ph * ni] = v; };
        const long long chunks = cdiv(n, kSegChunk);
        const long long seg = std::max(1LL, cdiv(chunks, 8LL * c.seg_chunks));
        const long long cellb = cdiv(nb, 256);
        set(BP_ZERO, cdiv(3 * nb, 1024));
        set(BP_KEY, I.cellsort ? cdiv(n, (long long)kSortThreads * kKeyItems) : I.ntiles);
        set(BP_SCAN0_R, I.scan0.nblk[0] + I.scan0.nblk[1]);
        set(BP_SCAN0_D, I.scan0.nblk[0] + I.scan0.nblk[1]);
        set(BP_SCAT0, I.cellsort ? 0 : I.ntiles);
        set(BP_HIST1, I.npasses == 2 ? I.ntiles : 0);
        set(BP_SCAN1_R, I.scan1.nblk[0]);
        set(BP_SCAN1_D, I.scan1.nblk[0]);
        set(BP_SCAT1, I.npasses == 2 ? I.ntiles : 0);
        set(BP_PLACE, I.cellsort ? cdiv(n, 512LL * kPlaceItems) : 0);
        set(BP_SEGSORT, I.cellsort ? cdiv(nb, (long long)kGroupCells * kSegSortWarps) : 0);
        set(BP_DEPV, seg);
        set(BP_AVG, std::max(1LL, cdiv(nb, 256LL * c.avg_items)));
        set(BP_PACK, cellb);
        set(BP_DRAG, std::max(1LL, cdiv(n, 256LL * c.drag_items)));
        set(BP_DEPM, seg);
        set(BP_PROJ, cellb);
        set(BP_PROJE, I.eps_fine ? cellb : 0);
        set(BP_SUMS, CG_NSUMS);
        // partial regions (pairs): volume 1 column, projection 6 (S_f V_f, S_B V_B), drag 9
        I.part_blocks[PS_VOL] = seg;
        I.part_blocks[PS_PROJ] = cellb;
        I.part_blocks[PS_DRAG] = B[(size_t)BP_DRAG * ni];
        I.part_off[PS_VOL] = 0;
        I.part_off[PS_PROJ] = seg;
        I.part_off[PS_DRAG] = seg + 6 * cellb;
        const long long pairs = I.part_off[PS_DRAG] + (long long)kDragSums * I.part_blocks[PS_DRAG];
        CG_TRY(dev_alloc(b, (void**)&I.part, sizeof(float) * 2 * pairs));
        I.smap = sums_map(I.part_off, I.part_blocks);
        if (!I.cellsort) {
            smem_key = std::max(smem_key, sizeof(int) << I.b0);
            smem_s0 = std::max(smem_s0, scatter_smem_bytes(I.b0, sizeof(float)));
        }
        if (I.npasses == 2) smem_s1 = std::max(smem_s1, scatter_smem_bytes(I.b1, sizeof(float)));
        if (I.npasses == 2) smem_hist1 = std::max(smem_hist1, sizeof(int) << I.b1);
    }
    // prefixes and persistent grids
    b->start.assign((size_t)BP_COUNT * (ni + 1), 0);
    for (int ph = 0; ph < BP_COUNT; ++ph) {
        long long acc = 0;
        for (int i = 0; i < ni; ++i) {
            b->start[(size_t)ph * (ni + 1) + i] = acc;
            acc += blocks[(size_t)ph * ni + i];
        }
        b->start[(size_t)ph * (ni + 1) + ni] = acc;
        b->total[ph] = acc;
    }
    b->smem[BP_KEY] = smem_key;
    b->smem[BP_HIST1] = smem_hist1;
    b->smem[BP_SCAT0] = smem_s0;
    b->smem[BP_SCAT1] = smem_s1;
    for (int ph = 0; ph < BP_COUNT; ++ph) {
        int occ = 1;
        switch (ph) {
            case BP_KEY: case BP_SCAN0_R: case BP_SCAN0_D: case BP_SCAT0:
            case BP_HIST1: case BP_SCAN1_R: case BP_SCAN1_D: case BP_SCAT1: case BP_PLACE: case BP_SEGSORT:
                occ = batch_bin_occupancy(ph, b->smem[ph]);
                break;
            case BP_AVG: case BP_PROJ: case BP_PROJE: occ = batch_fine_occupancy(ph); break;
            case BP_DRAG: occ = batch_drag_occupancy(); break;
            default: occ = batch_deposit_occupancy(ph); break;
        }
        const long long cap = (long long)occ * b->num_sms * c.grid_mult;
        b->grid[ph] = (unsigned)std::min(b->total[ph], cap);
    }
    void* di = nullptr;
    void* ds = nullptr;
    if (cudaMalloc(&di, sizeof(BInst) * ni) != cudaSuccess || cudaMalloc(&ds, sizeof(long long) * b->start.size()) != cudaSuccess) {
        cudaGetLastError();
        if (di) cudaFree(di);
        return CG_ERR_OOM;
    }
    b->d_inst = (BInst*)di;
    b->d_start = (long long*)ds;
    CG_CUDA(cudaMemcpy(b->d_inst, b->hi.data(), sizeof(BInst) * ni, cudaMemcpyHostToDevice));
    CG_CUDA(cudaMemcpy(b->d_start, b->start.data(), sizeof(long long) * b->start.size(), cudaMemcpyHostToDevice));
    return CG_OK;
}

// The launches of one batched step on the batch's stream.
cg_status enqueue(cg_batch* b, double dt) {
    const int ni = (int)b->h.size();
    auto L = [&](int ph) {
        BLaunch l;
        l.inst = b->d_inst;
        l.start = b->d_start + (size_t)ph * (ni + 1);
        l.ninst = ni;
        l.total = b->total[ph];
        return l;
    };
    cudaStream_t s = b->stream;
    for (int ph = 0; ph < BP_COUNT; ++ph) {
        if (b->total[ph] == 0) continue;
        switch (ph) {
            case BP_ZERO: case BP_DEPV: case BP_PACK: case BP_DEPM: case BP_SUMS:
                CG_TRY(launch_batch_deposit(ph, L(ph), b->grid[ph], s));
                break;
            case BP_AVG: case BP_PROJ: case BP_PROJE:
                CG_TRY(launch_batch_fine(ph, L(ph), b->grid[ph], s));
                break;
            case BP_DRAG:
                CG_TRY(launch_batch_drag(L(ph), b->grid[ph], (float)dt, s));
                break;
            default:
                CG_TRY(launch_batch_bin(ph, L(ph), b->grid[ph], b->smem[ph], s));
                break;
        }
        b->launches++;
    }
    return CG_OK;
}

// The reference sequence: cg_step of every instance in turn, each on its
// own handle with its own default launch shapes.
cg_status enqueue_each(cg_batch* b, double dt) {
    for (size_t i = 0; i < b->h.size(); ++i) {
        const cg_batch_item& it = b->items[i];
        CG_TRY(cg_step(b->h[i], &it.particles, it.u_fine, &it.out, dt));
    }
    return CG_OK;
}

// Run fn on the batch stream, through a captured graph (kept in *exec for
// this dt) when graphs are on.
template <typename Fn>
cg_status run_maybe_graph(cg_batch* b, cudaGraphExec_t* exec, double* exec_dt, double dt, Fn fn) {
    if (!b->use_graph) return fn();
    if (!*exec || *exec_dt != dt) {
        if (*exec) cudaGraphExecDestroy(*exec);
        *exec = nullptr;
        cudaGraph_t graph = nullptr;
        CG_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const cg_status st = fn();
        const cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
        if (st != CG_OK || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return st != CG_OK ? st : CG_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            *exec = nullptr;
            cudaGetLastError();
            return CG_ERR_CUDA;
        }
        *exec_dt = dt;
    }
    CG_CUDA(cudaGraphLaunch(*exec, b->stream));
    return CG_OK;
}

long long launches_per_step(const cg_batch* b) {
    long long k = 0;
    for (int ph = 0; ph < BP_COUNT; ++ph) k += b->total[ph] > 0;
    return k;
}

}  // namespace

extern "C" {

cg_status cg_batch_default_config(cg_batch_config* c) {
    if (!c) return CG_ERR_INVALID_ARG;
    c->digit_bits = kMaxDigitBits;
    c->drag_items = 1;
    c->avg_items = 1;
    c->seg_chunks = 1;
    c->grid_mult = 1;
    return CG_OK;
}

cg_status cg_batch_create(const cg_batch_item* items, int32_t count, void* cuda_stream, cg_batch** out) {
    if (!out) return CG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!items || count < 1 || count > 65536) return CG_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        const cg_batch_item& it = items[i];
        const cg_grid_desc& d = it.desc;
        if (d.prec != CG_FP32 || (d.ratio != 2 && d.ratio != 4 && d.ratio != 8)) return CG_ERR_INVALID_ARG;
        if (it.particles.n < 1 || it.particles.n > INT32_MAX || !it.particles.pos_d || !it.particles.vel)
            return CG_ERR_INVALID_ARG;
        if ((((uintptr_t)it.particles.pos_d) | ((uintptr_t)it.particles.vel)) & 15u) return CG_ERR_INVALID_ARG;
        const cg_step_out& o = it.out;
        if (!it.u_fine || !o.eps_bulk || !o.u_bulk || !o.S_bulk || !o.force || !o.S_fine) return CG_ERR_INVALID_ARG;
        if (o.cell || o.perm || o.cell_start || o.implicit_bulk || o.implicit_fine) return CG_ERR_INVALID_ARG;
        if ((((uintptr_t)it.u_fine) | ((uintptr_t)o.S_fine) | ((uintptr_t)o.eps_fine)) & 15u)
            return CG_ERR_INVALID_ARG;
    }
    cg_batch* b = new (std::nothrow) cg_batch();
    if (!b) return CG_ERR_OOM;
    b->user = (cudaStream_t)cuda_stream;
    cg_batch_default_config(&b->cfg);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    cg_status st = CG_OK;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess)
        st = CG_ERR_CUDA;
    b->items.assign(items, items + count);
    for (int i = 0; i < count && st == CG_OK; ++i) {
        cg_grids* g = nullptr;
        st = cg_create_grids(&items[i].desc, (void*)b->stream, &g);
        if (st != CG_OK) break;
        b->h.push_back(g);
        st = ensure_particle_capacity(g, items[i].particles.n);
    }
    if (st == CG_OK) st = plan(b);
    if (st != CG_OK) {
        cg_batch_destroy(b);
        return st;
    }
    *out = b;
    return CG_OK;
}

cg_status cg_batch_destroy(cg_batch* b) {
    if (!b) return CG_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    free_owned(b);
    for (cg_grids* g : b->h) cg_destroy_grids(g);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
    return CG_OK;
}

cg_status cg_batch_set_config(cg_batch* b, const cg_batch_config* c) {
    if (!b || !c || !valid_config(*c)) return CG_ERR_INVALID_ARG;
    CG_CUDA(cudaStreamSynchronize(b->stream));
    const cg_batch_config keep = b->cfg;
    b->cfg = *c;
    cg_status st = plan(b);
    if (st != CG_OK) {
        b->cfg = keep;
        cg_status st2 = plan(b);
        return st2 == CG_OK ? st : st2;
    }
    return CG_OK;
}

cg_status cg_batch_get_config(const cg_batch* b, cg_batch_config* c) {
    if (!b || !c) return CG_ERR_INVALID_ARG;
    *c = b->cfg;
    return CG_OK;
}

cg_status cg_batch_use_graph(cg_batch* b, int32_t on) {
    if (!b) return CG_ERR_INVALID_ARG;
    if (!on) drop_graph(b);
    b->use_graph = on != 0;
    return CG_OK;
}

cg_status cg_batch_step(cg_batch* b, double dt) {
    if (!b || !(dt >= 0.0) || !isfinite(dt)) return CG_ERR_INVALID_ARG;
    CG_CUDA(cudaEventRecord(b->ev_in, b->user));
    CG_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    const long long before = b->launches;
    CG_TRY(run_maybe_graph(b, &b->gexec, &b->graph_dt, dt, [&] { return enqueue(b, dt); }));
    b->launches = before + launches_per_step(b);
    CG_CUDA(cudaEventRecord(b->ev_out, b->stream));
    CG_CUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return CG_OK;
}

cg_status cg_batch_step_each(cg_batch* b, double dt) {
    if (!b || !(dt >= 0.0) || !isfinite(dt)) return CG_ERR_INVALID_ARG;
    CG_CUDA(cudaEventRecord(b->ev_in, b->user));
    CG_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    CG_TRY(run_maybe_graph(b, &b->gexec_each, &b->graph_dt_each, dt, [&] { return enqueue_each(b, dt); }));
    CG_CUDA(cudaEventRecord(b->ev_out, b->stream));
    CG_CUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return CG_OK;
}

cg_status cg_batch_sync_status(cg_batch* b, uint32_t* flags, int64_t* counts) {
    if (!b) return CG_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return CG_ERR_CUDA;
    }
    uint32_t f = 0;
    int64_t c[CG_NCOUNTS] = {0};
    cg_status worst = CG_OK;
    for (cg_grids* g : b->h) {
        uint32_t fi = 0;
        int64_t ci[CG_NCOUNTS] = {0};
        const cg_status s = cg_sync_status(g, &fi, ci);
        if (s == CG_ERR_CUDA) return s;
        if (worst == CG_OK) worst = s;
        f |= fi;
        for (int k = 0; k < CG_NCOUNTS; ++k) c[k] += ci[k];
    }
    if (flags) *flags = f;
    if (counts)
        for (int k = 0; k < CG_NCOUNTS; ++k) counts[k] = c[k];
    return worst;
}

cg_grids* cg_batch_instance(cg_batch* b, int32_t i) {
    if (!b || i < 0 || i >= (int32_t)b->h.size()) return nullptr;
    return b->h[i];
}

int64_t cg_batch_launch_count(const cg_batch* b) { return b ? b->launches : -1; }

int64_t cg_batch_launches_per_step(const cg_batch* b) { return b ? launches_per_step(b) : -1; }

// Autotuner: coordinate search over the decomposition knobs, each candidate
// timed (CUDA events on the batch stream, median of reps steps with dt = 0,
// so the particles do not move).  A cache file, when given, maps the batch
// signature (instance grids and particle counts) to its chosen
// configuration; a hit skips the search.
cg_status cg_batch_tune(cg_batch* b, int32_t reps, const char* cache_path, cg_batch_config* chosen,
                        double* best_ms) {
    if (!b || reps < 1 || reps > 1000) return CG_ERR_INVALID_ARG;
    std::string sig = "cgb1";
    for (size_t i = 0; i < b->items.size(); ++i) {
        const cg_batch_item& it = b->items[i];
        char buf[160];
        snprintf(buf, sizeof buf, ";%d,%d,%d,%d,%lld,%d,%d", it.desc.fine_n[0], it.desc.fine_n[1], it.desc.fine_n[2],
                 it.desc.ratio, (long long)it.particles.n, it.out.eps_fine ? 1 : 0, it.out.var_bulk ? 1 : 0);
        sig += buf;
    }
    if (cache_path) {
        FILE* f = fopen(cache_path, "r");
        if (f) {
            std::string line;
            char chunk[4096];
            cg_batch_config hit;
            bool found = false;
            while (fgets(chunk, sizeof chunk, f)) {
                line += chunk;
                if (line.empty() || line.back() != '\n') continue;
                const size_t sp = line.find(' ');
                if (sp != std::string::npos && line.compare(0, sp, sig) == 0 &&
                    sscanf(line.c_str() + sp + 1, "%d %d %d %d %d", &hit.digit_bits, &hit.drag_items, &hit.avg_items,
                           &hit.seg_chunks, &hit.grid_mult) == 5 &&
                    valid_config(hit))
                    found = true, b->cfg = hit;
                line.clear();
            }
            fclose(f);
            if (found) {
                CG_TRY(plan(b));
                if (chosen) *chosen = b->cfg;
                if (best_ms) *best_ms = -1.0;
                return CG_OK;
            }
        }
    }
    cudaEvent_t e0, e1;
    CG_CUDA(cudaEventCreate(&e0));
    CG_CUDA(cudaEventCreate(&e1));
    const bool graph = b->use_graph;
    b->use_graph = false;
    auto measure = [&](const cg_batch_config& c, double& ms) -> cg_status {
        b->cfg = c;
        CG_TRY(plan(b));
        CG_TRY(enqueue(b, 0.0));   // warm-up
        std::vector<float> t;
        for (int r = 0; r < reps; ++r) {
            CG_CUDA(cudaEventRecord(e0, b->stream));
            CG_TRY(enqueue(b, 0.0));
            CG_CUDA(cudaEventRecord(e1, b->stream));
            CG_CUDA(cudaEventSynchronize(e1));
            float x = 0.f;
            CG_CUDA(cudaEventElapsedTime(&x, e0, e1));
            t.push_back(x);
        }
        std::sort(t.begin(), t.end());
        ms = t[t.size() / 2];
        return CG_OK;
    };
    cg_batch_config best = b->cfg;
    double best_t = 0.0;
    cg_status st = measure(best, best_t);
    const int digit[] = {8, 9, 10, 11};
    const int items[] = {1, 2, 4, 8};
    const int mult[] = {1, 2, 4};
    for (int knob = 0; knob < 5 && st == CG_OK; ++knob) {
        const int* vals = knob == 0 ? digit : knob == 4 ? mult : items;
        const int nv = knob == 0 ? 4 : knob == 4 ? 3 : 4;
        for (int v = 0; v < nv && st == CG_OK; ++v) {
            cg_batch_config c = best;
            int* field = knob == 0 ? &c.digit_bits : knob == 1 ? &c.drag_items : knob == 2 ? &c.avg_items
                         : knob == 3 ? &c.seg_chunks : &c.grid_mult;
            if (*field == vals[v]) continue;
            *field = vals[v];
            double tm = 0.0;
            const cg_status s2 = measure(c, tm);
            if (s2 == CG_ERR_OUT_OF_RANGE) continue;   // digit too small for an instance
            st = s2;
            if (st == CG_OK && tm < best_t) {
                best_t = tm;
                best = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cfg = best;
    const cg_status sp = plan(b);
    b->use_graph = graph;
    if (st != CG_OK) return st;
    CG_TRY(sp);
    if (cache_path) {
        FILE* f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s %d %d %d %d %d\n", sig.c_str(), best.digit_bits, best.drag_items, best.avg_items,
                    best.seg_chunks, best.grid_mult);
            fclose(f);
        }
    }
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = best_t;
    return CG_OK;
}

}  // extern "C"
