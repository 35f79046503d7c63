// batch.cuh -- many independent coupling instances in one set of launches.
//
// A batched step runs each phase of the coupling step (zeroing, binning
// passes, porosity, fine -> bulk average, pack, drag, reaction, projections,
// sums) as ONE persistent launch over every instance: the grid is sized to
// the resident CTAs of the GPU and each CTA walks a list of virtual blocks,
// virtual block v belonging to instance i when start[i] <= v < start[i+1].
// The phase bodies are the same device functions as the one-instance
// kernels, called with the virtual block's coordinates, so a batched
// instance computes exactly what cg_step computes for it.  Phase boundaries
// are launch boundaries: no CTA ever waits on another.
#pragma once

#include "cg_internal.cuh"
#include "drag_law.cuh"

namespace cg {

// Device record of one FP32 instance: geometry, caller buffers and the
// handle's scratch.
struct BInst {
    GridDev gd;
    Phys<float> P;
    long long n;
    int ntiles, b0, b1, npasses;
    int cellsort;          // per-cell sort (else the digit sort)
    float* pos;
    float* vel;
    const float* u_fine;
    // outputs (cg_step_out of the instance)
    double* eps;
    float* u_bulk;
    float* var;
    float* S_bulk;
    float* force;
    float* S_fine;
    float* eps_fine;
    double* sums;
    // scratch of the instance's handle and of the batch
    int32_t* key;
    int32_t* count;        // cell counts, then cell_start after the scan
    int32_t* hist;
    int32_t* key1;         // digit sort: keys after pass 1; per-cell sort: second id buffer
    int32_t* val1;         // digit sort: ids after pass 1; per-cell sort: placed ids
    int32_t* arrival;      // per-cell sort: arrival rank in the cell
    int32_t* perm;
    int32_t* key_sorted;
    int32_t* inv_perm;
    int32_t* scan_part;
    float* vol;
    float* vol_sorted;
    float* Fs;
    float* bulk4;
    float* eps_t;
    float* part;                 // compensated partial pairs of this instance
    long long part_off[PS_NREG];
    long long part_blocks[PS_NREG];
    ScanJob scan0, scan1;
    SumsMap smap;
    unsigned long long* status;
};

// Phases of a batched step, in launch order.
enum BPhase {
    BP_ZERO = 0, BP_KEY, BP_SCAN0_R, BP_SCAN0_D, BP_SCAT0, BP_HIST1, BP_SCAN1_R, BP_SCAN1_D, BP_SCAT1,
    BP_PLACE, BP_SEGSORT, BP_DEPV, BP_AVG, BP_PACK, BP_DRAG, BP_DEPM, BP_PROJ, BP_PROJE, BP_SUMS, BP_COUNT
};

// One batched launch: virtual-block prefix over the instances (device).
struct BLaunch {
    const BInst* inst;
    const long long* start;   // [ninst + 1]
    int ninst;
    long long total;
};

// Instance owning virtual block v (start is non-decreasing, start[0] = 0,
// start[ninst] = total > v).
__device__ __forceinline__ int find_inst(const long long* __restrict__ start, int ninst, long long v) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Walk the virtual blocks of a launch; body(inst, blk) runs with the whole
// CTA, which synchronises before its shared memory is reused.
template <typename Body>
__device__ __forceinline__ void batch_loop(const BLaunch& L, Body body) {
    for (long long v = blockIdx.x; v < L.total; v += gridDim.x) {
        const int i = find_inst(L.start, L.ninst, v);
        const long long s0 = __ldg(L.start + i), s1 = __ldg(L.start + i + 1);
        body(L.inst[i], Blk{v - s0, s1 - s0});
        __syncthreads();
    }
}

// Launchers of the batched phases (one per source file that owns the body).
// grid: persistent CTAs; smem: dynamic shared memory per CTA.
cg_status launch_batch_bin(int phase, const BLaunch& L, unsigned grid, size_t smem, cudaStream_t s);
cg_status launch_batch_deposit(int phase, const BLaunch& L, unsigned grid, cudaStream_t s);
cg_status launch_batch_fine(int phase, const BLaunch& L, unsigned grid, cudaStream_t s);
cg_status launch_batch_drag(const BLaunch& L, unsigned grid, float dt, cudaStream_t s);
// Resident CTAs per SM of a phase's kernel.
int batch_bin_occupancy(int phase, size_t smem);
int batch_deposit_occupancy(int phase);
int batch_fine_occupancy(int phase);
int batch_drag_occupancy();

}  // namespace cg
