// map.cu -- maps between two uniform grids in any relative position and
// with any spacings: the grid-to-grid transfer of arXiv 1807.11834
// (Fig. 1 arrows; Sec. 2.3: the mapping structure is static and computed
// once per simulation) for grids that are not nested.
//
// With V(B & f) the volume of the intersection of bulk cell B and fine
// cell f:
//   average (fine -> bulk):  u_B = sum_f V(B & f) u_f / sum_f V(B & f)
//   project (bulk -> fine):  S_f = sum_B V(B & f) S_B / V_f   (conserves sum S V
//                            where the fine grid covers the bulk one)
// Both grids are boxes, so V(B & f) is the product of the overlaps of the
// cells' intervals on the three axes.  The static structure is one
// compressed-row table per axis and direction (bulk index -> overlapping
// fine indices and overlap lengths, and fine -> bulk), built once on the
// host in double and kept on the device; the 3-D weight of a pair is the
// product of its three axis entries.  Average: one thread per bulk cell
// walks its fine box (consecutive threads read consecutive fine runs);
// projection: when no fine cell overlaps more than two bulk cells along an
// axis (fine cells no larger than bulk cells) a fixed 2 x 2 x 2 stencil,
// one CTA per fine row with the bulk rows it reaches collapsed over y and z
// in shared memory first; else one thread per fine cell through the
// compressed rows.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "cg_internal.cuh"

struct cg_map {
    cg_box_grid bulk, fine;
    int fp64 = 0;
    size_t tsize = 4;
    cudaStream_t stream = nullptr;
    long long nbulk = 0, nfine = 0;
    // per axis: [ptr (n+1) int32][idx int32][w T], average (bulk rows) and projection (fine rows)
    void* dev = nullptr;
    long long off_bptr[3], off_bidx[3], off_bw[3], off_fptr[3], off_fidx[3], off_fw[3], off_cov[3];
    // when no fine cell overlaps more than two bulk cells along any axis:
    // per axis and fine index, the first bulk index and the two overlaps
    bool two = false;
    long long off_f2b[3], off_f2w0[3], off_f2w1[3];
    double Vf = 0.0;
};

namespace cg {
namespace {

// Cell bounds along an axis: x0 + i L / n (the same expression for the upper
// bound of cell i and the lower bound of cell i + 1).
inline double bound(const cg_box_grid& G, int a, long long i) { return G.origin[a] + (double)i * (G.extent[a] / G.n[a]); }

inline double overlap_len(double a0, double a1, double b0, double b1) {
    const double lo = std::max(a0, b0), hi = std::min(a1, b1);
    return hi > lo ? hi - lo : 0.0;
}

// Compressed rows of grid R's cells along axis a: for each row cell, the
// cells of grid C along a that overlap it, and the overlap lengths.
void axis_rows(const cg_box_grid& R, const cg_box_grid& Cg, int a, std::vector<int>& ptr, std::vector<int>& idx,
               std::vector<double>& w) {
    const int nr = R.n[a], nc = Cg.n[a];
    const double hc = Cg.extent[a] / nc;
    ptr.assign(nr + 1, 0);
    idx.clear();
    w.clear();
    for (int i = 0; i < nr; ++i) {
        const double lo = bound(R, a, i), hi = bound(R, a, i + 1);
        long long j0 = (long long)floor((lo - Cg.origin[a]) / hc) - 1, j1 = (long long)floor((hi - Cg.origin[a]) / hc) + 1;
        j0 = std::max(j0, 0LL);
        j1 = std::min(j1, (long long)nc - 1);
        for (long long j = j0; j <= j1; ++j) {
            const double v = overlap_len(lo, hi, bound(Cg, a, j), bound(Cg, a, j + 1));
            if (v > 0.0) {
                idx.push_back((int)j);
                w.push_back(v);
            }
        }
        ptr[i + 1] = (int)idx.size();
    }
}

template <typename T>
struct MapDev {
    const int* bptr[3];
    const int* bidx[3];
    const T* bw[3];
    const int* fptr[3];
    const int* fidx[3];
    const T* fw[3];
    const T* cov[3];   // per bulk index: covered length along the axis
    const int* f2b[3];
    const T* f2w0[3];
    const T* f2w1[3];
    int nb[3], nf[3];
    T inv_Vf;
};

template <typename T>
MapDev<T> dev_view(const cg_map* m) {
    MapDev<T> d;
    const char* base = (const char*)m->dev;
    for (int a = 0; a < 3; ++a) {
        d.bptr[a] = (const int*)(base + m->off_bptr[a]);
        d.bidx[a] = (const int*)(base + m->off_bidx[a]);
        d.bw[a] = (const T*)(base + m->off_bw[a]);
        d.fptr[a] = (const int*)(base + m->off_fptr[a]);
        d.fidx[a] = (const int*)(base + m->off_fidx[a]);
        d.fw[a] = (const T*)(base + m->off_fw[a]);
        d.cov[a] = (const T*)(base + m->off_cov[a]);
        d.f2b[a] = m->two ? (const int*)(base + m->off_f2b[a]) : nullptr;
        d.f2w0[a] = m->two ? (const T*)(base + m->off_f2w0[a]) : nullptr;
        d.f2w1[a] = m->two ? (const T*)(base + m->off_f2w1[a]) : nullptr;
        d.nb[a] = m->bulk.n[a];
        d.nf[a] = m->fine.n[a];
    }
    d.inv_Vf = (T)(1.0 / m->Vf);
    return d;
}

constexpr int kMapMaxComp = 8;

// Both kernels take cells in x-fastest order with 32-bit index arithmetic
// (grids hold fewer than 2^31 cells): one division per cell splits the index
// into the x index and the row (y, z), whose two axis ranges are looked up
// once per cell.
template <typename T, int NC>
__global__ void __launch_bounds__(256) k_map_average(MapDev<T> d, const T* __restrict__ in, T* __restrict__ out) {
    pdl_wait();
    const unsigned nbx = (unsigned)d.nb[0], nby = (unsigned)d.nb[1];
    const unsigned nbk = nbx * nby * (unsigned)d.nb[2];
    const unsigned nfx = (unsigned)d.nf[0], nfy = (unsigned)d.nf[1];
    const size_t nfn = (size_t)nfx * nfy * (unsigned)d.nf[2];
    for (unsigned cb = blockIdx.x * blockDim.x + threadIdx.x; cb < nbk; cb += gridDim.x * blockDim.x) {
        const unsigned row = cb / nbx;
        const unsigned I = cb - row * nbx;
        const unsigned J = row % nby, K = row / nby;
        const int x0 = __ldg(d.bptr[0] + I), x1 = __ldg(d.bptr[0] + I + 1);
        const int y0 = __ldg(d.bptr[1] + J), y1 = __ldg(d.bptr[1] + J + 1);
        const int z0 = __ldg(d.bptr[2] + K), z1 = __ldg(d.bptr[2] + K + 1);
        // each fine row's few x terms in plain FMAs, the row sums (weighted
        // by y and z) into compensated sums
        CSum<T> acc[NC];
        for (int kz = z0; kz < z1; ++kz) {
            const unsigned fz = (unsigned)__ldg(d.bidx[2] + kz);
            const T wz = __ldg(d.bw[2] + kz);
            for (int ky = y0; ky < y1; ++ky) {
                const unsigned fy = (unsigned)__ldg(d.bidx[1] + ky);
                const T wyz = __ldg(d.bw[1] + ky) * wz;
                const T* rowp = in + (size_t)nfx * (fy + nfy * fz);
                T rs[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) rs[c] = T(0);
                for (int kx = x0; kx < x1; ++kx) {
                    const unsigned fx = (unsigned)__ldg(d.bidx[0] + kx);
                    const T wx = __ldg(d.bw[0] + kx);
#pragma unroll
                    for (int c = 0; c < NC; ++c) rs[c] = fma(wx, __ldg(rowp + c * nfn + fx), rs[c]);
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[c].add(wyz * rs[c]);
            }
        }
        const T W = __ldg(d.cov[0] + I) * __ldg(d.cov[1] + J) * __ldg(d.cov[2] + K);
#pragma unroll
        for (int c = 0; c < NC; ++c) out[(size_t)c * nbk + cb] = W > T(0) ? acc[c].get() / W : T(0);
    }
}

template <typename T, int NC>
__global__ void __launch_bounds__(256) k_map_project(MapDev<T> d, const T* __restrict__ in, T* __restrict__ out) {
    pdl_wait();
    const unsigned nbx = (unsigned)d.nb[0], nby = (unsigned)d.nb[1];
    const size_t nbk = (size_t)nbx * nby * (unsigned)d.nb[2];
    const unsigned nfx = (unsigned)d.nf[0], nfy = (unsigned)d.nf[1];
    const unsigned nfn = nfx * nfy * (unsigned)d.nf[2];
    for (unsigned cf = blockIdx.x * blockDim.x + threadIdx.x; cf < nfn; cf += gridDim.x * blockDim.x) {
        const unsigned row = cf / nfx;
        const unsigned i = cf - row * nfx;
        const unsigned j = row % nfy, k = row / nfy;
        const int x0 = __ldg(d.fptr[0] + i), x1 = __ldg(d.fptr[0] + i + 1);
        const int y0 = __ldg(d.fptr[1] + j), y1 = __ldg(d.fptr[1] + j + 1);
        const int z0 = __ldg(d.fptr[2] + k), z1 = __ldg(d.fptr[2] + k + 1);
        T acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = T(0);
        for (int kz = z0; kz < z1; ++kz) {
            const unsigned bz = (unsigned)__ldg(d.fidx[2] + kz);
            const T wz = __ldg(d.fw[2] + kz);
            for (int ky = y0; ky < y1; ++ky) {
                const unsigned by = (unsigned)__ldg(d.fidx[1] + ky);
                const T wyz = __ldg(d.fw[1] + ky) * wz;
                const size_t brow = (size_t)nbx * (by + nby * bz);
                for (int kx = x0; kx < x1; ++kx) {
                    const size_t b = brow + (unsigned)__ldg(d.fidx[0] + kx);
                    const T w = __ldg(d.fw[0] + kx) * wyz;
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc[c] = fma(w, __ldg(in + c * nbk + b), acc[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) out[(size_t)c * nfn + cf] = acc[c] * d.inv_Vf;
    }
}

// Projection when every fine cell overlaps at most two bulk cells per axis:
// a fixed 2 x 2 x 2 stencil (the second weight 0 where there is one), all
// loads independent, as in the trilinear projection of nested grids.
template <typename T, int NC>
__global__ void __launch_bounds__(256) k_map_project2(MapDev<T> d, const T* __restrict__ in, T* __restrict__ out) {
    pdl_wait();
    const unsigned nbx = (unsigned)d.nb[0], nby = (unsigned)d.nb[1], nbz = (unsigned)d.nb[2];
    const size_t nbk = (size_t)nbx * nby * nbz;
    const unsigned nfx = (unsigned)d.nf[0], nfy = (unsigned)d.nf[1];
    const unsigned nfn = nfx * nfy * (unsigned)d.nf[2];
    for (unsigned cf = blockIdx.x * blockDim.x + threadIdx.x; cf < nfn; cf += gridDim.x * blockDim.x) {
        const unsigned row = cf / nfx;
        const unsigned i = cf - row * nfx;
        const unsigned j = row % nfy, k = row / nfy;
        const unsigned bx = (unsigned)__ldg(d.f2b[0] + i), by = (unsigned)__ldg(d.f2b[1] + j);
        const unsigned bz = (unsigned)__ldg(d.f2b[2] + k);
        const T wx[2] = {__ldg(d.f2w0[0] + i), __ldg(d.f2w1[0] + i)};
        const T wy[2] = {__ldg(d.f2w0[1] + j), __ldg(d.f2w1[1] + j)};
        const T wz[2] = {__ldg(d.f2w0[2] + k), __ldg(d.f2w1[2] + k)};
        // the second neighbour stays inside the grid (its weight is 0 at the edge)
        const unsigned dx = bx + 1 < nbx ? 1u : 0u, dy = by + 1 < nby ? nbx : 0u;
        const size_t dz = bz + 1 < nbz ? (size_t)nbx * nby : 0;
        const size_t b0 = bx + (size_t)nbx * (by + (size_t)nby * bz);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const T* s = in + c * nbk + b0;
            const T v000 = __ldg(s), v001 = __ldg(s + dx), v010 = __ldg(s + dy), v011 = __ldg(s + dy + dx);
            const T v100 = __ldg(s + dz), v101 = __ldg(s + dz + dx), v110 = __ldg(s + dz + dy);
            const T v111 = __ldg(s + dz + dy + dx);
            const T y0 = wy[0] * fma(wx[1], v001, wx[0] * v000) + wy[1] * fma(wx[1], v011, wx[0] * v010);
            const T y1 = wy[0] * fma(wx[1], v101, wx[0] * v100) + wy[1] * fma(wx[1], v111, wx[0] * v110);
            out[(size_t)c * nfn + cf] = (wz[0] * y0 + wz[1] * y1) * d.inv_Vf;
        }
    }
}

// Row-tiled projection (the default for the two-point stencil when its
// shared memory, NC x (bulk cells per x row) values, fits).  (A row-tiled
// average that collapsed the fine rows of each bulk row first read the fine
// field about 1.6 times over, and ran slower than the cell kernel above.)
// Projection with the two-point stencil: the CTA takes fine row (j, k); it
// first collapses the (at most 2 x 2) bulk rows over y and z for every bulk
// x index the row reaches, into shared memory, then thread i combines the
// two x neighbours of its fine cell.
template <typename T, int NC>
__global__ void __launch_bounds__(256) k_map_project2_rows(MapDev<T> d, const T* __restrict__ in, T* __restrict__ out) {
    pdl_wait();
    extern __shared__ unsigned char smem_raw[];
    T* v = reinterpret_cast<T*>(smem_raw);   // [NC][nbx]
    const unsigned nbx = (unsigned)d.nb[0], nby = (unsigned)d.nb[1], nbz = (unsigned)d.nb[2];
    const size_t nbk = (size_t)nbx * nby * nbz;
    const unsigned nfx = (unsigned)d.nf[0], nfy = (unsigned)d.nf[1];
    const unsigned nfn = nfx * nfy * (unsigned)d.nf[2];
    const unsigned rows = nfy * (unsigned)d.nf[2];
    for (unsigned r = blockIdx.x; r < rows; r += gridDim.x) {
        const unsigned j = r % nfy, k = r / nfy;
        const unsigned by = (unsigned)__ldg(d.f2b[1] + j), bz = (unsigned)__ldg(d.f2b[2] + k);
        const T wy0 = __ldg(d.f2w0[1] + j), wy1 = __ldg(d.f2w1[1] + j);
        const T wz0 = __ldg(d.f2w0[2] + k), wz1 = __ldg(d.f2w1[2] + k);
        const size_t dy = by + 1 < nby ? nbx : 0, dz = bz + 1 < nbz ? (size_t)nbx * nby : 0;
        const size_t b0 = (size_t)nbx * (by + (size_t)nby * bz);
        for (unsigned X = threadIdx.x; X < nbx; X += blockDim.x) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const T* s = in + c * nbk + b0 + X;
                v[c * nbx + X] = wz0 * fma(wy1, __ldg(s + dy), wy0 * __ldg(s)) +
                                 wz1 * fma(wy1, __ldg(s + dz + dy), wy0 * __ldg(s + dz));
            }
        }
        __syncthreads();
        for (unsigned i = threadIdx.x; i < nfx; i += blockDim.x) {
            const unsigned bx = (unsigned)__ldg(d.f2b[0] + i);
            const unsigned bx1 = bx + 1 < nbx ? bx + 1 : bx;
            const T wx0 = __ldg(d.f2w0[0] + i), wx1 = __ldg(d.f2w1[0] + i);
            const unsigned cf = i + nfx * r;
#pragma unroll
            for (int c = 0; c < NC; ++c) out[(size_t)c * nfn + cf] = fma(wx1, v[c * nbx + bx1], wx0 * v[c * nbx + bx]) * d.inv_Vf;
        }
        __syncthreads();
    }
}

bool finite3(const double* v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

bool valid_box(const cg_box_grid& G) {
    if (!finite3(G.origin) || !finite3(G.extent)) return false;
    for (int a = 0; a < 3; ++a)
        if (!(G.extent[a] > 0.0) || G.n[a] < 1) return false;
    const long long n = (long long)G.n[0] * G.n[1] * G.n[2];
    return n <= 2147483647LL && (G.prec == CG_FP32 || G.prec == CG_FP64);
}

unsigned grid_for(long long m) { return (unsigned)std::max(1LL, std::min((m + 255) / 256, 1LL << 16)); }

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" cg_status cg_map_create(const cg_box_grid* bulk, const cg_box_grid* fine, void* cuda_stream,
                                   cg_map** out) {
    if (!out) return CG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!bulk || !fine || !valid_box(*bulk) || !valid_box(*fine) || bulk->prec != fine->prec) return CG_ERR_INVALID_ARG;
    cg_map* m = new (std::nothrow) cg_map();
    if (!m) return CG_ERR_OOM;
    m->bulk = *bulk;
    m->fine = *fine;
    m->fp64 = bulk->prec == CG_FP64;
    m->tsize = m->fp64 ? 8 : 4;
    m->stream = (cudaStream_t)cuda_stream;
    m->nbulk = (long long)bulk->n[0] * bulk->n[1] * bulk->n[2];
    m->nfine = (long long)fine->n[0] * fine->n[1] * fine->n[2];
    m->Vf = (fine->extent[0] / fine->n[0]) * (fine->extent[1] / fine->n[1]) * (fine->extent[2] / fine->n[2]);
    // host tables, then one device block: per axis, bulk rows, fine rows, covered lengths
    std::vector<int> bp[3], bi[3], fp[3], fi[3];
    std::vector<double> bw[3], fw[3], cov[3];
    for (int a = 0; a < 3; ++a) {
        axis_rows(*bulk, *fine, a, bp[a], bi[a], bw[a]);
        axis_rows(*fine, *bulk, a, fp[a], fi[a], fw[a]);
        cov[a].assign(bulk->n[a], 0.0);
        for (int i = 0; i < bulk->n[a]; ++i)
            for (int k = bp[a][i]; k < bp[a][i + 1]; ++k) cov[a][i] += bw[a][k];
    }
    std::vector<unsigned char> host;
    auto put = [&](const void* p, size_t bytes) {
        const long long off = (long long)((host.size() + 255) & ~(size_t)255);
        host.resize((size_t)off + bytes);
        if (bytes) memcpy(host.data() + off, p, bytes);
        return off;
    };
    auto put_t = [&](const std::vector<double>& v) {
        if (m->fp64) return put(v.data(), v.size() * sizeof(double));
        std::vector<float> f(v.begin(), v.end());
        return put(f.data(), f.size() * sizeof(float));
    };
    m->two = true;
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < fine->n[a]; ++i) m->two = m->two && fp[a][i + 1] - fp[a][i] <= 2;
    for (int a = 0; a < 3 && m->two; ++a) {
        std::vector<int> b0(fine->n[a], 0);
        std::vector<double> w0(fine->n[a], 0.0), w1(fine->n[a], 0.0);
        for (int i = 0; i < fine->n[a]; ++i) {
            const int k0 = fp[a][i], k1 = fp[a][i + 1];
            if (k1 > k0) {
                b0[i] = fi[a][k0];
                w0[i] = fw[a][k0];
                if (k1 - k0 == 2) w1[i] = fw[a][k0 + 1];
            }
        }
        m->off_f2b[a] = put(b0.data(), b0.size() * sizeof(int));
        m->off_f2w0[a] = put_t(w0);
        m->off_f2w1[a] = put_t(w1);
    }
    for (int a = 0; a < 3; ++a) {
        m->off_bptr[a] = put(bp[a].data(), bp[a].size() * sizeof(int));
        m->off_bidx[a] = put(bi[a].data(), bi[a].size() * sizeof(int));
        m->off_bw[a] = put_t(bw[a]);
        m->off_fptr[a] = put(fp[a].data(), fp[a].size() * sizeof(int));
        m->off_fidx[a] = put(fi[a].data(), fi[a].size() * sizeof(int));
        m->off_fw[a] = put_t(fw[a]);
        m->off_cov[a] = put_t(cov[a]);
    }
    if (cudaMalloc(&m->dev, std::max<size_t>(host.size(), 16)) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return CG_ERR_OOM;
    }
    if (cudaMemcpy(m->dev, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(m->dev);
        delete m;
        return CG_ERR_CUDA;
    }
    *out = m;
    return CG_OK;
}

extern "C" cg_status cg_map_destroy(cg_map* m) {
    if (!m) return CG_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    else cudaDeviceSynchronize();
    cudaFree(m->dev);
    delete m;
    return CG_OK;
}

// The map's launches go through CG_LAUNCH's counterpart without a handle:
// a programmatic dependent launch on the map's stream.
template <typename K, typename... Args>
static cg_status map_launch(cg_map* m, K kernel, long long work, Args... args) {
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t c = {};
    c.gridDim = dim3(grid_for(work));
    c.blockDim = dim3(256);
    c.stream = m->stream;
    c.attrs = a;
    c.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&c, kernel, args...);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

constexpr size_t kMapRowSmem = 96 * 1024;   // shared memory of a row-tiled CTA at most

template <typename K>
static cg_status row_attr(K kernel, size_t smem) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMapRowSmem) != cudaSuccess) {
        cudaGetLastError();
        return CG_ERR_CUDA;
    }
    return CG_OK;
}

// One CTA per row (grid-stride over the rows), with dynamic shared memory.
template <typename K, typename... Args>
static cg_status map_launch_rows(cg_map* m, K kernel, long long rows, size_t smem, Args... args) {
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t c = {};
    c.gridDim = dim3((unsigned)std::max(1LL, std::min(rows, 65535LL)));
    c.blockDim = dim3(256);
    c.dynamicSmemBytes = smem;
    c.stream = m->stream;
    c.attrs = a;
    c.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&c, kernel, args...);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

template <typename T, int NC>
static cg_status map_apply(cg_map* m, bool avg, const void* in, void* out) {
    if (avg) return map_launch(m, k_map_average<T, NC>, m->nbulk, dev_view<T>(m), (const T*)in, (T*)out);
    if (m->two) {
        const size_t smem = (size_t)NC * m->bulk.n[0] * sizeof(T);
        if (smem <= kMapRowSmem) {
            CG_TRY(row_attr(k_map_project2_rows<T, NC>, smem));
            return map_launch_rows(m, k_map_project2_rows<T, NC>, (long long)m->fine.n[1] * m->fine.n[2], smem,
                                   dev_view<T>(m), (const T*)in, (T*)out);
        }
        return map_launch(m, k_map_project2<T, NC>, m->nfine, dev_view<T>(m), (const T*)in, (T*)out);
    }
    return map_launch(m, k_map_project<T, NC>, m->nfine, dev_view<T>(m), (const T*)in, (T*)out);
}

template <typename T>
static cg_status map_dispatch(cg_map* m, bool avg, int ncomp, const void* in, void* out) {
    switch (ncomp) {
        case 1: return map_apply<T, 1>(m, avg, in, out);
        case 2: return map_apply<T, 2>(m, avg, in, out);
        case 3: return map_apply<T, 3>(m, avg, in, out);
        case 4: return map_apply<T, 4>(m, avg, in, out);
        case 5: return map_apply<T, 5>(m, avg, in, out);
        case 6: return map_apply<T, 6>(m, avg, in, out);
        case 7: return map_apply<T, 7>(m, avg, in, out);
        case 8: return map_apply<T, 8>(m, avg, in, out);
    }
    return CG_ERR_INVALID_ARG;
}

static bool aligned_for(const cg_map* m, const void* p) { return ((uintptr_t)p & (m->tsize - 1)) == 0; }

extern "C" cg_status cg_map_average(cg_map* m, int32_t ncomp, const void* fine_in, void* bulk_out) {
    if (!m || ncomp < 1 || ncomp > kMapMaxComp || !fine_in || !bulk_out) return CG_ERR_INVALID_ARG;
    if (!aligned_for(m, fine_in) || !aligned_for(m, bulk_out)) return CG_ERR_INVALID_ARG;
    return m->fp64 ? map_dispatch<double>(m, true, ncomp, fine_in, bulk_out)
                   : map_dispatch<float>(m, true, ncomp, fine_in, bulk_out);
}

extern "C" cg_status cg_map_project(cg_map* m, int32_t ncomp, const void* bulk_in, void* fine_out) {
    if (!m || ncomp < 1 || ncomp > kMapMaxComp || !bulk_in || !fine_out) return CG_ERR_INVALID_ARG;
    if (!aligned_for(m, bulk_in) || !aligned_for(m, fine_out)) return CG_ERR_INVALID_ARG;
    return m->fp64 ? map_dispatch<double>(m, false, ncomp, bulk_in, fine_out)
                   : map_dispatch<float>(m, false, ncomp, bulk_in, fine_out);
}
