// static_bin.cu -- particle binning for callers that cannot allocate device
// memory.
//
// Some callers of this library must not call cudaMalloc: code that runs
// while another component is capturing a CUDA graph, plug-ins that may only
// touch the memory their host application hands them, and codes that budget
// every device byte through their own allocator.  cg_bin_particles_static
// serves them.  It bins like cg_bin_particles but needs no handle: all its
// scratch lives in one file-scope device array of fixed size, and its
// outputs go to the caller's buffers.  It allocates nothing and frees
// nothing.
//
// The array below is part of the library's device image: every GPU that
// loads the library holds it (about 12 MB) until the process exits.  Host
// code cannot use the array's name as a device address; the address is
// looked up once per device with cudaGetSymbolAddress on the first call
// made with that device current.  Make that first call before any stream
// capture begins.  Every call uses the same array, so calls whose work
// overlaps on the GPU (different streams, or different host threads) race
// and corrupt each other's results; order them on one stream.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "cg_internal.cuh"

namespace {

constexpr long long kStaticMaxParticles = 1LL << 18;   // 262,144
constexpr long long kStaticMaxTiles = kStaticMaxParticles / cg::kSortTile;
constexpr long long kStaticHist = kStaticMaxTiles << cg::kMaxDigitBits;
constexpr long long kStaticScanPart =
    (kStaticHist + cg::kScanItems - 1) / cg::kScanItems +
    ((1LL << cg::kMaxBulkBits) + 1 + cg::kScanItems - 1) / cg::kScanItems + 2;

// Scratch layout (byte offsets, each region 256-byte aligned).
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffKey = 0;
constexpr size_t kOffKey1 = kOffKey + align256(4 * kStaticMaxParticles);
constexpr size_t kOffVal1 = kOffKey1 + align256(4 * kStaticMaxParticles);
constexpr size_t kOffKey2 = kOffVal1 + align256(4 * kStaticMaxParticles);
constexpr size_t kOffVal2 = kOffKey2 + align256(4 * kStaticMaxParticles);
constexpr size_t kOffKeySorted = kOffVal2 + align256(4 * kStaticMaxParticles);
constexpr size_t kOffInvPerm = kOffKeySorted + align256(4 * kStaticMaxParticles);
constexpr size_t kOffVol = kOffInvPerm + align256(4 * kStaticMaxParticles);
constexpr size_t kOffVolSorted = kOffVol + align256(8 * kStaticMaxParticles);
constexpr size_t kOffHist = kOffVolSorted + align256(8 * kStaticMaxParticles);
constexpr size_t kOffScan = kOffHist + align256(4 * kStaticHist);
constexpr size_t kOffStatus = kOffScan + align256(4 * kStaticScanPart);
constexpr size_t kStaticBytes = kOffStatus + align256(sizeof(unsigned long long) * cg::kNumSlots);

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

namespace {

std::mutex g_addr_mu;
void* g_addr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
cg_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return CG_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CG_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return CG_OK;
}

bool finite3(const double* v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

}  // namespace

extern "C" cg_status cg_bin_particles_static(const cg_grid_desc* desc, int64_t n, const void* pos_d,
                                             int32_t* cell_out, int32_t* perm_out, int32_t* cell_start_out,
                                             void* cuda_stream) {
    if (!desc || !perm_out || !cell_start_out) return CG_ERR_INVALID_ARG;
    if (n < 0) return CG_ERR_INVALID_ARG;
    if (n > kStaticMaxParticles) return CG_ERR_OUT_OF_RANGE;
    if (n > 0 && (!pos_d || ((uintptr_t)pos_d & 15u))) return CG_ERR_INVALID_ARG;
    const cg_grid_desc& d = *desc;
    if (!finite3(d.origin) || !finite3(d.extent) || d.ratio < 1) return CG_ERR_INVALID_ARG;
    if (d.prec != CG_FP32 && d.prec != CG_FP64) return CG_ERR_INVALID_ARG;
    long long nbulk = 1;
    int nb[3];
    for (int a = 0; a < 3; ++a) {
        if (!(d.extent[a] > 0.0) || d.fine_n[a] < 1 || d.fine_n[a] % d.ratio != 0) return CG_ERR_INVALID_ARG;
        nb[a] = d.fine_n[a] / d.ratio;
        if (nb[a] < 2) return CG_ERR_INVALID_ARG;
        // refuse before the product can overflow: each factor is at most
        // 2^22, so the running product stays below 2^63
        if (nb[a] > (1 << cg::kMaxBulkBits)) return CG_ERR_OUT_OF_RANGE;
        nbulk *= nb[a];
        if (nbulk > (1LL << cg::kMaxBulkBits)) return CG_ERR_OUT_OF_RANGE;
    }
    if (!cg::sort_choice_valid(d.sort_digits)) return CG_ERR_INVALID_ARG;
    if (nbulk > (1LL << cg::kMaxBulkBits)) return CG_ERR_OUT_OF_RANGE;

    void* base = nullptr;
    CG_TRY(scratch_address(&base));
    unsigned char* s = (unsigned char*)base;

    // A handle on the host stack: geometry of the bin rule and pointers into
    // the static scratch; constructing it allocates nothing on the device.
    cg_grids g;
    g.desc = d;
    g.fp64 = d.prec == CG_FP64;
    g.tsize = g.fp64 ? 8 : 4;
    g.stream = (cudaStream_t)cuda_stream;
    cg::GridDev& gd = g.gd;
    memset(&gd, 0, sizeof gd);
    gd.r = d.ratio;
    gd.nbulk = nbulk;
    gd.nfine = (long long)d.fine_n[0] * d.fine_n[1] * d.fine_n[2];
    for (int a = 0; a < 3; ++a) {
        gd.nb[a] = nb[a];
        gd.nf[a] = d.fine_n[a];
        gd.x0[a] = d.origin[a];
        gd.xhi[a] = d.origin[a] + d.extent[a];
        gd.H[a] = d.extent[a] / (double)nb[a];
        gd.invH[a] = 1.0 / gd.H[a];
        gd.x0f[a] = (float)d.origin[a];
        gd.invHf[a] = (float)gd.invH[a];
        gd.ax0f[a] = (float)fabs(d.origin[a] * gd.invH[a]);
    }
    int bits = 0;
    while ((1LL << bits) < nbulk) ++bits;
    bits = std::max(bits, 1);
    g.npasses = cg::split_passes(bits, g.pass_bits, d.sort_digits >= 6 ? d.sort_digits : 0);
    g.key = (int32_t*)(s + kOffKey);
    g.key1 = (int32_t*)(s + kOffKey1);
    g.val1 = (int32_t*)(s + kOffVal1);
    g.key2 = (int32_t*)(s + kOffKey2);
    g.val2 = (int32_t*)(s + kOffVal2);
    g.key_sorted = (int32_t*)(s + kOffKeySorted);
    g.inv_perm = (int32_t*)(s + kOffInvPerm);
    g.vol = s + kOffVol;
    g.vol_sorted = s + kOffVolSorted;
    g.hist = (int32_t*)(s + kOffHist);
    g.scan_part = (int32_t*)(s + kOffScan);
    g.status = (unsigned long long*)(s + kOffStatus);
    g.hist_cap = kStaticHist;
    g.scan_cap = kStaticScanPart;
    g.cap = kStaticMaxParticles;
    g.perm = perm_out;
    g.cell_start = cell_start_out;   // the per-cell counts are accumulated here and scanned in place

    CG_TRY(cg::launch_bin(&g, n, pos_d));
    if (cell_out && n > 0)
        CG_CUDA(cudaMemcpyAsync(cell_out, g.key, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, g.stream));
    return CG_OK;
}
