// Allocation-free neighbour counting.
//
// Some callers cannot allocate device memory for us: a host solver or plugin
// framework that owns every device byte through its own pool and hands this
// library only its particle buffers, or a real-time loop that must not
// allocate after start-up (cudaMalloc may synchronise the device and has no
// latency bound).  For them dem_neighbor_counts_noalloc runs the cell binning
// of the neighbour-list build without any workspace: its scratch lives in one
// fixed, file-scope device array that every GPU loading this library holds
// until the process exits.
#include "dem.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

namespace cgdem {
void set_thread_error(const std::string& msg);
}

namespace {

constexpr long long NA_MAX_PARTICLES = 1ll << 18;   // 262,144
constexpr long long NA_MAX_CELLS = 1ll << 18;       // 262,144
// layout: pos int4[NP] | cell u32[NP] | slot u32[NP] | sorted u32[NP] | count u32[NC] | start u32[NC]
constexpr size_t NA_BYTES = (size_t)NA_MAX_PARTICLES * (16 + 4 + 4 + 4) + (size_t)NA_MAX_CELLS * (4 + 4);

static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

struct NaGrid {
    int ext[3], per[3], half[3], nc[3];
    int skin;
    int n;
    int ncell;
};

struct NaScratch {
    int4* pos;
    unsigned* cell;
    unsigned* slot;
    unsigned* sorted;
    unsigned* count;
    unsigned* start;
};

NaScratch carve(unsigned char* base)
{
    NaScratch s;
    s.pos = (int4*)base;
    s.cell = (unsigned*)(base + NA_MAX_PARTICLES * 16);
    s.slot = s.cell + NA_MAX_PARTICLES;
    s.sorted = s.slot + NA_MAX_PARTICLES;
    s.count = s.sorted + NA_MAX_PARTICLES;
    s.start = s.count + NA_MAX_CELLS;
    return s;
}

__device__ __forceinline__ int na_axis_cell(const NaGrid& g, int a, int x)
{
    if (x <= 0) return 0;
    long long t = (long long)x * g.nc[a] / g.ext[a];
    return t >= g.nc[a] ? g.nc[a] - 1 : (int)t;
}

__device__ __forceinline__ int na_min_image(int dx, int per, int L, int half)
{
    if (per) {
        if (dx > half) dx -= L;
        else if (dx < -half) dx += L;
    }
    return dx;
}

__global__ void k_na_clear(NaScratch s, NaGrid g)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) s.count[c] = 0u;
}

// Same rounding as dem_write: u = rint((x - lo) / q), wrapped into [0, L) on periodic axes.
__global__ void k_na_bin(NaScratch s, NaGrid g, const double* __restrict__ x, const double* __restrict__ r,
                         double lo0, double lo1, double lo2, double q)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const double lo[3] = {lo0, lo1, lo2};
    int u[3];
    for (int a = 0; a < 3; ++a) {
        double v = rint((x[3 * i + a] - lo[a]) / q);
        if (g.per[a]) {
            const double L = (double)g.ext[a];
            v = v - L * floor(v / L);
            if (v >= L) v -= L;
        }
        v = fmin(fmax(v, -2.0e9), 2.0e9);
        u[a] = (int)v;
    }
    const int4 p = make_int4(u[0], u[1], u[2], (int)rint(r[i] / q));
    s.pos[i] = p;
    const unsigned c = (unsigned)((na_axis_cell(g, 2, p.z) * g.nc[1] + na_axis_cell(g, 1, p.y)) * g.nc[0] +
                                  na_axis_cell(g, 0, p.x));
    s.cell[i] = c;
    s.slot[i] = atomicAdd(&s.count[c], 1u);
}

// exclusive scan of the cell counts in one block (ncell <= NA_MAX_CELLS)
__global__ void __launch_bounds__(1024) k_na_scan(NaScratch s, NaGrid g)
{
    __shared__ unsigned wsum[32];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c0 = 0; c0 < g.ncell; c0 += 1024) {
        const int c = c0 + threadIdx.x;
        const unsigned v = c < g.ncell ? s.count[c] : 0u;
        unsigned x = v;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned w = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const unsigned ex = carry + (warp ? wsum[warp - 1] : 0u) + x - v;
        if (c < g.ncell) s.start[c] = ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
}

__global__ void k_na_scatter(NaScratch s, NaGrid g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    s.sorted[s.start[s.cell[i]] + s.slot[i]] = (unsigned)i;
}

// neighbours j != i with |x_ij| < r_i + r_j + skin (exact integer test, minimum image)
__global__ void k_na_count(NaScratch s, NaGrid g, int* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int4 p = s.pos[i];
    const int cx0 = na_axis_cell(g, 0, p.x), cy0 = na_axis_cell(g, 1, p.y), cz0 = na_axis_cell(g, 2, p.z);
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        const int cz = cz0 + dz;
        if (cz < 0 || cz >= g.nc[2]) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int cy = cy0 + dy;
            if (cy < 0 || cy >= g.nc[1]) {
                if (!g.per[1]) continue;
                cy = (cy + g.nc[1]) % g.nc[1];
            }
            for (int dx = -1; dx <= 1; ++dx) {
                int cx = cx0 + dx;
                if (cx < 0 || cx >= g.nc[0]) {
                    if (!g.per[0]) continue;
                    cx = (cx + g.nc[0]) % g.nc[0];
                }
                const int c = (cz * g.nc[1] + cy) * g.nc[0] + cx;
                const unsigned b = s.start[c], e = b + s.count[c];
                for (unsigned t = b; t < e; ++t) {
                    const int j = (int)s.sorted[t];
                    if (j == i) continue;
                    const int4 q = s.pos[j];
                    const long long ddx = na_min_image(p.x - q.x, g.per[0], g.ext[0], g.half[0]);
                    const long long ddy = na_min_image(p.y - q.y, g.per[1], g.ext[1], g.half[1]);
                    const long long ddz = (long long)p.z - q.z;
                    const long long cut = (long long)p.w + q.w + g.skin;
                    // one axis at a time first (as the list build does): positions clamped far
                    // outside an open box must not overflow the sum of squares
                    if (llabs(ddx) >= cut || llabs(ddy) >= cut || llabs(ddz) >= cut) continue;
                    if (ddx * ddx + ddy * ddy + ddz * ddz < cut * cut) ++cnt;
                }
            }
        }
    }
    out[i] = cnt;
}

dem_status na_fail(dem_status st, const std::string& msg)
{
    cgdem::set_thread_error(msg);
    return st;
}

}  // namespace

extern "C" dem_status dem_neighbor_counts_noalloc(const double* x, const double* r, int64_t n, const double lo[3],
                                                  const double hi[3], const int32_t periodic[3], double skin,
                                                  double r_max, int32_t* counts, void* stream)
{
    if (n < 0 || !lo || !hi || !periodic || (n > 0 && (!x || !r || !counts)))
        return na_fail(DEM_ERR_ARG, "dem_neighbor_counts_noalloc: null argument or negative n");
    if (n > NA_MAX_PARTICLES)
        return na_fail(DEM_ERR_CAPACITY, "dem_neighbor_counts_noalloc: n exceeds the fixed maximum of 262144 particles");
    if (!(skin >= 0) || !(r_max > 0) || periodic[2])
        return na_fail(DEM_ERR_ARG, "dem_neighbor_counts_noalloc: need skin >= 0, r_max > 0, z not periodic");
    NaGrid g{};
    double ext[3], emax = 0.0;
    for (int a = 0; a < 3; ++a) {
        ext[a] = hi[a] - lo[a];
        if (!(ext[a] > 0)) return na_fail(DEM_ERR_ARG, "dem_neighbor_counts_noalloc: empty box");
        emax = std::fmax(emax, ext[a]);
    }
    // the same length quantum and integer units as a context (see dem.h)
    double q = std::ldexp(1.0, (int)std::ceil(std::log2(emax / 1073741824.0)));
    while (emax / q > 1073741824.0) q *= 2.0;
    const long long rmax_u = (long long)std::ceil(r_max / q);
    const long long skin_u = (long long)std::llround(skin / q);
    const long long hcell = 2 * rmax_u + skin_u;
    long long ncell = 1;
    for (int a = 0; a < 3; ++a) {
        const long long eu = std::llround(ext[a] / q);
        g.ext[a] = (int)eu;
        g.per[a] = periodic[a] ? 1 : 0;
        g.half[a] = (int)(eu / 2);
        long long nc = eu / hcell;
        if (g.per[a] && nc < 3)
            return na_fail(DEM_ERR_ARG, "dem_neighbor_counts_noalloc: periodic axis shorter than 3 cells");
        if (nc < 1) nc = 1;
        if (nc > NA_MAX_CELLS) nc = NA_MAX_CELLS;
        g.nc[a] = (int)nc;
        ncell *= nc;
    }
    if (ncell > NA_MAX_CELLS)
        return na_fail(DEM_ERR_CAPACITY, "dem_neighbor_counts_noalloc: cell grid exceeds the fixed maximum of 262144 cells");
    g.skin = (int)skin_u;
    g.n = (int)n;
    g.ncell = (int)ncell;
    if (n == 0) return DEM_OK;

    // the device address of the scratch array on the current device, looked up on every call
    // (cheap next to the launches; a cached address would outlive a device reset)
    void* base = nullptr;
    {
        cudaError_t e = cudaGetSymbolAddress(&base, g_na_scratch);
        if (e != cudaSuccess || !base)
            return na_fail(DEM_ERR_CUDA, std::string("dem_neighbor_counts_noalloc: cudaGetSymbolAddress: ") +
                                             cudaGetErrorString(e));
    }
    const NaScratch s = carve((unsigned char*)base);
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned nb = (unsigned)((n + 255) / 256);
    k_na_clear<<<(unsigned)std::min<long long>((ncell + 255) / 256, 1024), 256, 0, st>>>(s, g);
    k_na_bin<<<nb, 256, 0, st>>>(s, g, x, r, lo[0], lo[1], lo[2], q);
    k_na_scan<<<1, 1024, 0, st>>>(s, g);
    k_na_scatter<<<nb, 256, 0, st>>>(s, g);
    k_na_count<<<nb, 256, 0, st>>>(s, g, counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return na_fail(DEM_ERR_CUDA, std::string("dem_neighbor_counts_noalloc: launch: ") + cudaGetErrorString(e));
    return DEM_OK;
}
