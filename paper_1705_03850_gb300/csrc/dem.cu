// GB300 (sm_103a) kernels and C ABI of the DEM hot path: contact forces of
// Eqs. 3-6 with tangential history (Sec. 2.1), velocity Verlet of Eqs. 1-2,
// and device-side neighbour-list rebuilds.  See include/dem.h for the
// interface and dem_internal.cuh for the data layout.
#include "dem.h"
#include "dem_internal.cuh"
#include "dem_ctx.h"
#include "dem_contact.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace cgdem;

// minimum resident blocks per SM requested for the step kernel (register budget)
#ifndef DEM_STEP_MINB
#define DEM_STEP_MINB 7
#endif

// ====================================================================== scan
// Exclusive scan of the per-cell counts into cell starts: three passes over
// tiles of SCAN_TILE entries (per-tile sums, scan of the sums, tile scans).

namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_V = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_V;

__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* total)
{
    __shared__ unsigned wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (warp == 0) {
        unsigned w = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    unsigned base = warp ? wsum[warp - 1] : 0u;
    *total = wsum[nw - 1];
    __syncthreads();
    return base + x - v;
}

// A scan chunk belongs to one instance (code ranges are aligned to chunks);
// chunks of instances that are not rebuilding are skipped.
__device__ __forceinline__ bool chunk_active(const Dev& d, unsigned b)
{
    const int k = d.part_inst[b];
    return k >= 0 && d.id[k].flag != 0;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(Dev d)
{
    if (!d.g->any) return;
    const unsigned b = blockIdx.x;
    if (!chunk_active(d, b)) {
        if (threadIdx.x == 0) d.part[b] = 0u;
        return;
    }
    const unsigned base = b * SCAN_TILE;
    unsigned s = 0;
    for (int k = 0; k < SCAN_V; ++k) {
        unsigned i = base + k * SCAN_T + threadIdx.x;
        if (i < d.ncodes) s += d.ccount[i];
    }
    unsigned tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) d.part[b] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(Dev d)
{
    if (!d.g->any) return;
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (unsigned c0 = 0; c0 < d.nparts; c0 += blockDim.x) {
        unsigned i = c0 + threadIdx.x;
        unsigned v = i < d.nparts ? d.part[i] : 0u;
        unsigned tot;
        unsigned ex = block_exclusive_scan(v, &tot);
        if (i < d.nparts) d.part[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_down(Dev d)
{
    if (!d.g->any || !chunk_active(d, blockIdx.x)) return;
    const unsigned base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_V;
    unsigned v[SCAN_V];
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) {
        unsigned i = base + k;
        v[k] = i < d.ncodes ? d.ccount[i] : 0u;
        s += v[k];
    }
    unsigned tot;
    unsigned ex = block_exclusive_scan(s, &tot) + d.part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) {
        unsigned i = base + k;
        if (i < d.ncodes) d.crange[i] = make_uint2(ex, v[k]);
        ex += v[k];
    }
}

// ==================================================================== cells
// (axis_cell, cell_code, min_image in dem_internal.cuh)

// ================================================================ rebuild
// Triggered per instance by the displacement bound (flag != 0).  Sequence:
// clear counts -> bin (atomic slot in cell) -> scan -> scatter -> order each
// cell by particle ID -> count -> order the slots of each tile by contact count
// (and copy positions and IDs in cell order) -> build lists, permute state,
// carry histories -> finish.

// Per-slot rebuild work runs on a persistent grid of TILE-thread blocks that
// strides over the tiles and skips tiles of instances that are not rebuilding.
template <typename Fn>
__device__ __forceinline__ void for_rebuilding_slots(const Dev& d, Fn fn)
{
    for (int t = blockIdx.x; t < d.ntiles; t += gridDim.x) {
        const int k = d.tile_inst[t];
        const InstD D = d.id[k];
        if (!D.flag) continue;
        const InstC& c = d.ic[k];
        const int s = t * TILE + threadIdx.x;
        if (s - c.slot0 >= D.n) continue;
        fn(s, D, c);
    }
}

__global__ void k_rb_clear(Dev d)
{
    if (!d.g->any) return;
    for (unsigned b = blockIdx.x; b < d.nparts; b += gridDim.x) {
        if (!chunk_active(d, b)) continue;
        for (unsigned i = b * SCAN_TILE + threadIdx.x; i < (b + 1) * SCAN_TILE && i < d.ncodes; i += blockDim.x)
            d.ccount[i] = 0u;
    }
}

__global__ void __launch_bounds__(TILE) k_rb_bin(Dev d)
{
    if (!d.g->any) return;
    for_rebuilding_slots(d, [&](int s, const InstD& D, const InstC& c) {
        const unsigned idw = __float_as_uint(d.vel[D.cur][s].w);
        if (idw & GONE_BIT) {               // removed particle: not binned, its ID unmapped
            d.slot_of_id[c.slot0 + (int)(idw & ID_MASK)] = -1;
            d.cslot[s] = 0xffffffffu;
            return;
        }
        const int4 p = d.pos[D.cur][s];
        const unsigned code = cell_code(d, c, axis_cell(c, 0, p.x), axis_cell(c, 1, p.y), axis_cell(c, 2, p.z));
        d.cellcode[s] = code;
        d.cslot[s] = atomicAdd(&d.ccount[code], 1u);
    });
}

__global__ void __launch_bounds__(TILE) k_rb_scatter(Dev d)
{
    if (!d.g->any) return;
    for_rebuilding_slots(d, [&](int s, const InstD& D, const InstC& c) {
        if (d.cslot[s] == 0xffffffffu) return;   // removed
        const unsigned code = d.cellcode[s];
        const int np = c.slot0 + (int)(d.crange[code].x - d.crange[c.code0].x) + (int)d.cslot[s];
        d.perm[np] = s;
    });
}

// The first member of every cell orders the cell by particle ID, so that the
// final order depends only on the cells and the IDs.
__global__ void __launch_bounds__(TILE) k_rb_cellsort(Dev d)
{
    if (!d.g->any) return;
    for_rebuilding_slots(d, [&](int s, const InstD& D, const InstC& c) {
        if (d.cslot[s] != 0u) return;   // not the first of its cell, or removed
        const unsigned code = d.cellcode[s];
        const int cntc = (int)d.ccount[code];
        if (cntc < 2) return;
        int* a = d.perm + c.slot0 + (int)(d.crange[code].x - d.crange[c.code0].x);
        const float4* v = d.vel[D.cur];
        for (int i = 1; i < cntc; ++i) {
            const int x = a[i];
            const unsigned xid = __float_as_uint(v[x].w) & ID_MASK;
            int j = i - 1;
            while (j >= 0 && (__float_as_uint(v[a[j]].w) & ID_MASK) > xid) {
                a[j + 1] = a[j];
                --j;
            }
            a[j + 1] = x;
        }
    });
}

// Slots within each tile of TILE cell-order positions go to the particles in order
// of decreasing contact count at the last step (then list length, then cell
// order), so that the 32 rows a warp of the step kernel walks together have
// similar lengths.  Results do not depend on the slot order: every particle sums
// its own row in the row's order.  Also writes the cell-order copies of
// positions and IDs that the list build scans.  Results do not depend on the slot order: every particle sums
// its own row in the row's order.
__global__ void __launch_bounds__(TILE) k_rb_tilesort(Dev d)
{
    if (!d.g->any) return;
    __shared__ unsigned key[TILE];
    for (int t = blockIdx.x; t < d.ntiles; t += gridDim.x) {
        const int k = d.tile_inst[t];
        const InstD D = d.id[k];            // the same for the whole block
        if (!D.flag) continue;
        const InstC& c = d.ic[k];
        const int p = t * TILE + threadIdx.x;
        const int nvalid = min(TILE, D.n_new - (t * TILE - c.slot0));
        const bool valid = (int)threadIdx.x < nvalid;
        unsigned kk = 0u;
        if (valid) {
            const int old = d.perm[p];
            d.spos[p] = d.pos[D.cur][old];                    // cell-order copies for the list build
            d.sid[p] = (int)(__float_as_uint(d.vel[D.cur][old].w) & ID_MASK);
            if (D.flag != 2)
                kk = ((unsigned)__popc(d.hmask[D.lp][old]) << 8) | (unsigned)min(d.cnt[D.lp][old], 255);
        }
        __syncthreads();                    // the previous tile's keys are no longer read
        key[threadIdx.x] = kk;
        __syncthreads();
        if (valid) {
            int rank = 0;
            for (int j = 0; j < nvalid; ++j) {
                const unsigned kj = key[j];
                rank += (kj > kk || (kj == kk && j < (int)threadIdx.x)) ? 1 : 0;
            }
            const int s = t * TILE + rank;
            d.fin[p] = s;
        }
    }
}

// The same order over windows of at most SMW_SORT_W tiles, for the SM-wide step blocks (single
// instance): an SM's warps walk the slices of neighbouring tiles together, so a window of
// several tiles can be ordered as one and its 32-row slices come out more alike (the 1M bed's
// step kernel: 106.9 µs against 112.8 µs with windows of one tile; 108.5 µs with windows of 8
// tiles, 111.6 µs with 32, 121.7 µs with 64: wider windows spread a slice's rows over a
// larger region than the SM's warps walk at once; cut from the step blocks' shares, windows of
// at most 12, 16 and 18 tiles gave 99.1, 100.4 and 99.4 µs).  A stable counting sort
// on (contacts, list length), both at most MAXL: 256 threads per window, each warp ranks its
// run of 32-element chunks with __match_any_sync and counts per key, and the per-warp counts,
// scanned over the keys, give each warp's first rank per key.
#ifndef SMW_SORT_W
#define SMW_SORT_W 12
#endif
constexpr int WS_T = 256;                          // threads per window
constexpr int WS_KEYS = (MAXL + 1) * (MAXL + 1);   // (contacts, list length) pairs
template <int W>
__global__ void __launch_bounds__(WS_T) k_rb_winsort(Dev d, int G)
{
    constexpr int N = W * TILE;                    // slots per window
    constexpr int NW = WS_T / 32;                  // warps
    constexpr int PER = N / WS_T;                  // 32-element chunks per warp
    constexpr int BPT = (WS_KEYS + WS_T - 1) / WS_T;
    static_assert(N % WS_T == 0 && N <= 65535, "window of whole warp chunks, ranks in 16 bits");
    if (!d.g->any) return;
    __shared__ unsigned short hist[NW][WS_KEYS];   // per-warp counts per key, then first ranks
    __shared__ int wsum[NW];
    const int lane = (int)threadIdx.x & 31, w = (int)threadIdx.x >> 5;
    // the windows split each of the G step blocks' shares of the live tiles (the same split as
    // the step kernel's) into K parts of at most W tiles: a share's last slices, which its warps
    // claim last and the other SMs take over, are the lightest of its last window
    const InstD D = d.id[0];                // SM-wide blocks: a single instance
    if (!D.flag) return;
    const InstC& c = d.ic[0];
    const int tf = c.slot0 / TILE, nt = (D.n_new + TILE - 1) / TILE;
    const int K = max(1, ((nt + G - 1) / G + W - 1) / W);
    for (int wi = blockIdx.x; wi < G * K; wi += gridDim.x) {
        const int b = wi / K, kk = wi % K;
        const int s0 = (int)((long long)b * nt / G), len = (int)((long long)(b + 1) * nt / G) - s0;
        const int t0 = tf + s0 + len * kk / K, t1 = tf + s0 + len * (kk + 1) / K;
        const int p0 = t0 * TILE;
        const int nvalid = min((t1 - t0) * TILE, D.n_new - (p0 - c.slot0));
        if (nvalid <= 0) continue;
        __syncthreads();                    // the previous window's ranks are read
        for (int i = threadIdx.x; i < NW * WS_KEYS; i += WS_T) (&hist[0][0])[i] = 0;
        __syncthreads();
        int key[PER];
        unsigned short rk[PER];
#pragma unroll
        for (int cc = 0; cc < PER; ++cc) {
            const int i = w * PER * 32 + cc * 32 + lane;
            int kk = -1;
            if (i < nvalid) {
                const int p = p0 + i;
                const int old = d.perm[p];
                d.spos[p] = d.pos[D.cur][old];                    // cell-order copies for the list build
                d.sid[p] = (int)(__float_as_uint(d.vel[D.cur][old].w) & ID_MASK);
                kk = 0;
                if (D.flag != 2) {
                    const int nc = min(__popc(d.hmask[D.lp][old]), MAXL), nl = min(d.cnt[D.lp][old], MAXL);
                    kk = WS_KEYS - 1 - (nc * (MAXL + 1) + nl);    // more contacts, longer rows first
                }
            }
            const unsigned m = __match_any_sync(0xffffffffu, kk);
            const int below = __popc(m & ((1u << lane) - 1u));  // equal keys in earlier lanes
            rk[cc] = kk >= 0 ? (unsigned short)(hist[w][kk] + below) : (unsigned short)0;
            __syncwarp();
            if (kk >= 0 && below == 0) hist[w][kk] += (unsigned short)__popc(m);
            __syncwarp();
            key[cc] = kk;
        }
        __syncthreads();
        // each thread a run of BPT keys: totals, an exclusive scan over the block, then each
        // warp's first rank per key (keys in order, warps in order within a key)
        int tot[BPT];
        int run = 0;
#pragma unroll
        for (int j = 0; j < BPT; ++j) {
            const int b = (int)threadIdx.x * BPT + j;
            int tb = 0;
            if (b < WS_KEYS)
#pragma unroll
                for (int v = 0; v < NW; ++v) tb += hist[v][b];
            tot[j] = tb;
            run += tb;
        }
        int inc = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        int first = inc - run;
        for (int v = 0; v < w; ++v) first += wsum[v];
#pragma unroll
        for (int j = 0; j < BPT; ++j) {
            const int b = (int)threadIdx.x * BPT + j;
            if (b < WS_KEYS) {
                int o = first;
#pragma unroll
                for (int v = 0; v < NW; ++v) {
                    const int h = hist[v][b];
                    hist[v][b] = (unsigned short)o;
                    o += h;
                }
            }
            first += tot[j];
        }
        __syncthreads();
#pragma unroll
        for (int cc = 0; cc < PER; ++cc) {
            const int i = w * PER * 32 + cc * 32 + lane;
            if (i < nvalid) d.fin[p0 + i] = p0 + hist[w][key[cc]] + rk[cc];
        }
    }
}

// One thread per particle: move it into its new slot of the other state buffer,
// collect neighbours within r_i + r_j + skin (exact integer test), order the
// row by overlap depth, and carry the tangential overlaps of pairs that were
// already listed (found by ID in the particle's previous row).  The candidate
// row is kept in shared memory, entry-major so that the threads of a warp hit
// different banks.
constexpr int RB_T = 64;                     // threads per block of the list build

struct RowScratch {
    float key[MAXL][RB_T];                   // d^2 - (r_i + r_j)^2 (rounded to float: monotone)
    int pos[MAXL][RB_T];                     // partner's cell-order position
};

// The staged variant of the list build: the block's 64 cell-order positions and RB_W on either
// side (the cells around the block's particles, in Morton order) staged in shared memory;
// candidates inside the window are read from there, the others from L2.
constexpr int RB_W = 128;
constexpr int RB_WIN = RB_T + 2 * RB_W;
struct Window {
    int4 pos[RB_WIN];
    int lo, n;                               // first cell-order position and length
};

template <bool STAGED>
__device__ __forceinline__ void build_row(const Dev& d, int ps, const InstD& D, const InstC& c, RowScratch& R,
                                          const Window* W)
{
    const int tx = threadIdx.x;
    const int cur = D.cur, nxt = cur ^ 1, lp = D.lp, nlp = lp ^ 1;
    const int ncap = d.ncap;
    const int s = d.fin[ps];                // this particle's new slot
    const int old = d.perm[ps];
    const int4 p = d.pos[cur][old];
    float4 v = d.vel[cur][old];
    const float4 w = d.omg[cur][old];
    const unsigned myid = __float_as_uint(v.w) & ID_MASK;
    if (D.flag == 2) v.w = __uint_as_float(myid);   // fresh start: no floor history
    d.pos[nxt][s] = p;
    d.vel[nxt][s] = v;
    d.omg[nxt][s] = w;
    d.slot_of_id[c.slot0 + (int)myid] = s;

    // candidates ordered by (d^2 - (r_i + r_j)^2, ID): deepest overlaps first, so
    // that within a warp the contacts sit in the leading entries of every row
    int nc = 0;
    bool overflow = false;
    const int ccx = axis_cell(c, 0, p.x), ccy = axis_cell(c, 1, p.y), ccz = axis_cell(c, 2, p.z);
    const unsigned cbase = d.crange[c.code0].x;
    const int Lmax = d.Lmax;
    const int per0 = c.per[0], per1 = c.per[1], ext0 = c.ext[0], ext1 = c.ext[1], hf0 = c.half[0], hf1 = c.half[1];
    const int skin = c.skin;
    // the Morton parts of the (up to) three neighbour cells per axis (x and y wrap when
    // periodic, z never does) and a 27-bit mask of the cells that exist
    unsigned mx[3], my[3], mz[3];
    unsigned okm = 0u;
    {
        bool okx[3], oky[3], okz[3];
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            int cx = ccx + o - 1, cy = ccy + o - 1;
            const int cz = ccz + o - 1;
            okx[o] = oky[o] = true;
            if (cx < 0) { okx[o] = c.per[0] != 0; cx += c.nc[0]; }
            else if (cx >= c.nc[0]) { okx[o] = c.per[0] != 0; cx -= c.nc[0]; }
            if (cy < 0) { oky[o] = c.per[1] != 0; cy += c.nc[1]; }
            else if (cy >= c.nc[1]) { oky[o] = c.per[1] != 0; cy -= c.nc[1]; }
            okz[o] = cz >= 0 && cz < c.nc[2];
            mx[o] = okx[o] ? __ldg(d.spread + c.spread_off[0] + cx) : 0u;
            my[o] = oky[o] ? __ldg(d.spread + c.spread_off[1] + cy) : 0u;
            mz[o] = okz[o] ? __ldg(d.spread + c.spread_off[2] + cz) : 0u;
        }
#pragma unroll
        for (int k = 0; k < 27; ++k)
            if (okx[k % 3] && oky[(k / 3) % 3] && okz[k / 9]) okm |= 1u << k;
    }
    const unsigned mx0 = mx[0], mx1 = mx[1], mx2 = mx[2], my0 = my[0], my1 = my[1], my2 = my[2];
    const unsigned mz0 = mz[0], mz1 = mz[1], mz2 = mz[2];
    auto range_of = [&](int k) -> uint2 {
        if (!((okm >> k) & 1u)) return make_uint2(0u, 0u);
        const int ix = k % 3, iy = (k / 3) % 3, iz = k / 9;
        const unsigned code = (unsigned)c.code0 + (ix == 0 ? mx0 : ix == 1 ? mx1 : mx2) +
                              (iy == 0 ? my0 : iy == 1 ? my1 : my2) + (iz == 0 ? mz0 : iz == 1 ? mz1 : mz2);
#if DEM_CHECKS
        if (!in_range(d, (long long)code - c.code0, c.ncode, ps, 1)) return make_uint2(0u, 0u);
#endif
        return __ldg(d.crange + code);
    };
    // scan the 27 cells (the next cell's range in flight) and append the neighbours
    // within the skin to the row unsorted; the row is sorted once at the end
    uint2 rg = range_of(0);
#pragma unroll 1
    for (int k = 0; k < 27; ++k) {
        const uint2 cr = rg;
        if (k + 1 < 27) rg = range_of(k + 1);
        const int start = c.slot0 + (int)(cr.x - cbase);
#if DEM_CHECKS
        int cnt = (int)cr.y;
        // a cell's candidates lie within the instance's slots (a cell outside the grid reads as
        // empty, with no start)
        if (cnt > 0 &&
            !(in_range(d, start - c.slot0, c.cap, ps, 2) && in_range(d, start - c.slot0 + cnt, c.cap + 1, ps, 2)))
            cnt = 0;
#else
        // (the checks compiled out: even folded away they cost this kernel registers)
        const int cnt = (int)cr.y;
#endif
        for (int t = 0; t < cnt; ++t) {
            const int m = start + t;
            int4 q;
            if (STAGED) {
                const unsigned wi = (unsigned)(m - W->lo);
                q = wi < (unsigned)W->n ? W->pos[wi] : __ldg(d.spos + m);
            } else {
                q = __ldg(d.spos + m);
            }
            const int ddx = min_image(p.x - q.x, per0, ext0, hf0);
            const int ddy = min_image(p.y - q.y, per1, ext1, hf1);
            const long long ddz = (long long)p.z - q.z;
            const int cut = p.w + q.w + skin;
            // most candidates fail on one axis already (32-bit compares)
            if (abs(ddx) >= cut || abs(ddy) >= cut || ddz >= cut || ddz <= -cut || m == ps) continue;
            const long long d2 = (long long)ddx * ddx + (long long)ddy * ddy + ddz * ddz;
            if (d2 >= (long long)cut * cut) continue;
            const long long S = (long long)p.w + q.w;
            if (nc == Lmax) {
                overflow = true;
                continue;
            }
            R.key[nc][tx] = (float)(d2 - S * S);
            R.pos[nc][tx] = m;
            ++nc;
        }
    }
    // order the row by (key, ID): equal keys (rare) by ID, so that the row does not
    // depend on the scan order
    for (int i = 1; i < nc; ++i) {
        const float key = R.key[i][tx];
        const int m = R.pos[i][tx];
        int j = i - 1;
        while (j >= 0 && (R.key[j][tx] > key || (R.key[j][tx] == key && d.sid[R.pos[j][tx]] > d.sid[m]))) {
            R.key[j + 1][tx] = R.key[j][tx];
            R.pos[j + 1][tx] = R.pos[j][tx];
            --j;
        }
        R.key[j + 1][tx] = key;
        R.pos[j + 1][tx] = m;
    }
    if (overflow) {
        atomicOr(&d.g->status, ST_CAPACITY);
        d.g->err_slot = s;
    }
    int* nrow = d.nbr[nlp] + s;
    float* hn = d.hist[nlp] + s;
    const size_t plane = (size_t)Lmax * ncap;
    const int* orow = d.nbr[lp] + old;
    const float* ho = d.hist[lp] + old;
    // the new row (partner slots); the keys give way to the partner IDs.  Stored overlaps are
    // written only where carried: every reader of an entry's overlap first checks its bit in the
    // history mask, so the other entries' storage is never read
    for (int e = 0; e < nc; ++e) {
        const int m = R.pos[e][tx];
        nrow[(size_t)e * ncap] = d.fin[m];
        R.key[e][tx] = __int_as_float(d.sid[m]);
    }
    // carry every non-zero stored overlap of the old row to the pair's new entry
    const int ocnt = D.flag == 2 ? 0 : d.cnt[lp][old];
    unsigned ohm = D.flag == 2 ? 0u : d.hmask[lp][old];
    if (ocnt < 32) ohm &= (1u << ocnt) - 1u;
    unsigned nhm = 0u;
    while (ohm) {
        const int eo = __ffs(ohm) - 1;
        ohm &= ohm - 1u;
        const float hx = ho[(size_t)eo * ncap], hy = ho[plane + (size_t)eo * ncap], hz = ho[2 * plane + (size_t)eo * ncap];
        if (hx == 0.f && hy == 0.f && hz == 0.f) continue;
        const int oid = (int)(__float_as_uint(d.vel[cur][orow[(size_t)eo * ncap]].w) & ID_MASK);
        for (int e = 0; e < nc; ++e) {
            if (__float_as_int(R.key[e][tx]) == oid) {
                hn[(size_t)e * ncap] = hx;
                hn[plane + (size_t)e * ncap] = hy;
                hn[2 * plane + (size_t)e * ncap] = hz;
                nhm |= 1u << e;
                break;
            }
        }
    }
    d.cnt[nlp][s] = nc;
    d.hmask[nlp][s] = nhm;
    if (D.fext) d.fext[nlp][s] = d.fext[lp][old];      // held until overwritten, even across state writes
    d.whist[nlp][s] = D.flag == 2 ? make_float4(0.f, 0.f, 0.f, 0.f) : d.whist[lp][old];
    if (c.nwp >= 2) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        d.wseg[nlp][s] = D.flag == 2 ? z : d.wseg[lp][old];
        d.wseg[nlp][ncap + s] = D.flag == 2 ? z : d.wseg[lp][ncap + old];
    }
}

template <bool STAGED>
__global__ void __launch_bounds__(RB_T, 16) k_rb_build(Dev d)
{
    if (!d.g->any) return;
    __shared__ RowScratch R;
    constexpr int H = TILE / RB_T;           // blocks of RB_T threads per tile
    // over the cell-order positions: the threads of a warp hold neighbouring particles and
    // scan overlapping cells (the rows go to the particles' new slots in the same tile).  The
    // direct scan (the default) finds the neighbouring cells' positions in L1: staging them in
    // shared memory (STAGED) was measured slower (0.83 against 0.70 ms per build of the 1M bed)
    for (int u = blockIdx.x; u < d.ntiles * H; u += gridDim.x) {
        const int t = u / H;
        const int k = d.tile_inst[t];
        const InstD D = d.id[k];
        if (!D.flag) continue;               // the same for the whole block
        const InstC& c = d.ic[k];
        const int p0 = t * TILE + (u % H) * RB_T;
        const int p = p0 + threadIdx.x;
        if (STAGED) {
            __shared__ Window W;
            const int lo = max(c.slot0, p0 - RB_W), hi = min(c.slot0 + D.n_new, p0 + RB_T + RB_W);
            __syncthreads();                 // the previous window is no longer read
            if (threadIdx.x == 0) {
                W.lo = lo;
                W.n = max(0, hi - lo);
            }
            for (int i = lo + (int)threadIdx.x; i < hi; i += RB_T) W.pos[i - lo] = __ldg(d.spos + i);
            __syncthreads();
            if (p - c.slot0 < D.n_new) build_row<true>(d, p, D, c, R, &W);
        } else {
            if (p - c.slot0 >= D.n_new) continue;
            build_row<false>(d, p, D, c, R, nullptr);
        }
    }
}

// live particles after the rebuild: the binned ones (removed particles dropped)
__global__ void k_rb_count(Dev d)
{
    if (!d.g->any) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d.B; k += gridDim.x * blockDim.x) {
        InstD& D = d.id[k];
        if (!D.flag) continue;
        const InstC& c = d.ic[k];
        const unsigned last = (unsigned)(c.code0 + c.ncode - 1);
        D.n_new = (int)(d.crange[last].x + d.crange[last].y - d.crange[c.code0].x);
    }
}

__global__ void k_rb_finish(Dev d)
{
    if (!d.g->any) return;
    for (int k = threadIdx.x; k < d.B; k += blockDim.x) {
        InstD& D = d.id[k];
        if (D.flag) {
            D.cur ^= 1;
            D.lp ^= 1;
            D.flag = 0;
            D.n = D.n_new;
            D.nbin = D.n_new;
            D.disp = 0.f;
            atomicAdd(&d.g->rebuilds, 1ull);
        }
    }
    __syncthreads();
    // the tiles fused steps walk: per instance the pairs of tiles that hold its live slots
    // (offsets by a scan over a chunk of instances, then the chunk's ranges written by the block)
    __shared__ unsigned s_off[256], s_lt[256];
    __shared__ int s_t0[256];
    unsigned base = 0u;
    for (int k0 = 0; k0 < d.B; k0 += blockDim.x) {
        const int k = k0 + (int)threadIdx.x;
        unsigned lt = 0u;
        if (k < d.B) lt = 2u * (unsigned)((d.id[k].n + 2 * TILE - 1) / (2 * TILE));
        unsigned tot;
        const unsigned off = base + block_exclusive_scan(lt, &tot);
        s_off[threadIdx.x] = off;
        s_lt[threadIdx.x] = lt;
        s_t0[threadIdx.x] = k < d.B ? d.ic[k].slot0 / TILE : 0;
        __syncthreads();
        const int nk = min((int)blockDim.x, d.B - k0);
        for (int j = 0; j < nk; ++j)
            for (unsigned i = threadIdx.x; i < s_lt[j]; i += blockDim.x) d.live_tiles[s_off[j] + i] = s_t0[j] + (int)i;
        __syncthreads();
        base += tot;
    }
    if (threadIdx.x == 0) {
        d.g->nlive = (int)base;
        d.g->any = 0u;
    }
}

// ============================================================= contact law
// (contact_fwd / contact_vjp in dem_contact.cuh)

using V3 = Vec3<float>;
__device__ __forceinline__ V3 v3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ Coef<float> coef_of(const InstC& c)
{
    return Coef<float>{c.c_kn, c.c_kt, c.nbeta, c.gt_ratio, c.mu, c.mu_w, c.clamp_fn};
}

// ================================================================== step
// MODE 0: one velocity-Verlet step (force at x^n with v^{n-1/2}, merged kick,
// drift to x^{n+1}, displacement bound, rebuild decision by the last block).
// MODE 1: forces at the current state only, written to the output arrays.
//
// Persistent grid: block b owns the contiguous tile range [b T / G, (b+1) T / G)
// (neighbouring tiles share neighbours, which then hit in L1), one thread per
// particle.  The row is walked twice: first the positions of all entries (in
// batches of four, the next batch's indices in flight) give the touch mask, then
// only the contacts are evaluated, in row order, with the next contact's state in
// flight; the stored
// overlap is loaded only for entries whose history is non-zero (bit mask hmask),
// and stored only where it changes.  Each particle evaluates its contacts from its own side; the
// contact law has a single call site, so both particles of a pair run the same
// instructions on operands that differ only in the sign of the antisymmetric
// ones.
// 32-bit integer hash ("lowbias32", C. Wellons' hash-prospector search, public domain)
__device__ __forceinline__ unsigned mix32(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// |(x, y)| from x^2 + y^2 >= 0 in double: a float root refined by one Newton step (the float
// root is within 1e-7 of the result, so the step leaves an error of order 1e-14 relative), in
// place of a double square root, which is slow on this GPU
__device__ __forceinline__ double root_refined(double s2)
{
    if (!(s2 > 0.0)) return 0.0;
    const float rf = sqrtf((float)s2);
    const double rd = (double)rf;
    return rd + (double)((float)fma(-rd, rd, s2) * (0.5f / rf));
}

// Axisymmetric walls: the surface of revolution of the polyline (rho_i, z_i) about a vertical
// axis, one wall per segment with its end points included (a free rim is an edge contact).
// Each touching segment is a particle-wall contact of Eqs. 3-6 at rest, with the wall
// friction; n runs from the nearest point of the segment, in the particle's azimuthal
// half-plane, to the centre.  Distances are taken in double from the exact integer position
// (the overlap is a small difference of two lengths), for the segments a float pre-test
// leaves within a 1/64 radius of contact: along the segment's unit normal when the closest
// point is inside the segment, else to the end point, with no double division or square root.
// The tangential overlaps of up to two segment contacts are kept per particle, tagged with the
// segment; MODE 0 stores them.
template <int MODE>
__device__ __forceinline__ int wall_contacts(const Dev& d, const InstC& c, int kinst, int s, int lp, int4 P, float r,
                                             float m, V3 vme, V3 wme, float dt_hist, V3& F, V3& Tq)
{
    const float exf = (float)(P.x - c.waxi) - c.waxf, eyf = (float)(P.y - c.wayi) - c.wayf, zf = (float)P.z;
    const float rhof = sqrtf(exf * exf + eyf * eyf);
    const float tol = 1e-6f * (rhof + fabsf(zf) + c.wmag) + 4.f;
    const float lim = (float)P.w * (1.f + 1.f / 64.f) + tol;
    const WallGeo& G = d.wgeo[kinst];
    unsigned nearm = 0u;
    for (int k = 0; k + 1 < c.nwp; ++k) {
        const float r0 = c.wpf[2 * k], z0 = c.wpf[2 * k + 1];
        const float dr = c.wpf[2 * k + 2] - r0, dz = c.wpf[2 * k + 3] - z0;
        const float t = fminf(fmaxf(((rhof - r0) * dr + (zf - z0) * dz) * G.inv2[k], 0.f), 1.f);
        const float a = rhof - (r0 + t * dr), b = zf - (z0 + t * dz);
        if (a * a + b * b < lim * lim) nearm |= 1u << k;
    }
    float4* ws = d.wseg[lp];
    const size_t ncap = (size_t)d.ncap;
    int nst = 0;
    if (nearm) {
        const float4 h0 = ws[s], h1 = ws[ncap + s];
        const double ex = (double)P.x - c.wax, ey = (double)P.y - c.way, z = (double)P.z;
        const double rho = root_refined(fma(ex, ex, ey * ey));
        float erx = 1.f, ery = 0.f;   // radial direction (float suffices for a direction)
        if (rhof > 0.f) {
            erx = exf / rhof;
            ery = eyf / rhof;
        }
        while (nearm) {
            const int k = __ffs(nearm) - 1;
            nearm &= nearm - 1u;
            // offset (a, b) of the centre from the segment's closest point, and its length
            const double ur = G.ur[k], uz = G.uz[k], len = G.len[k];
            const double pr = rho - c.wp[2 * k], pz = z - c.wp[2 * k + 1];
            const double sp = fma(pr, ur, pz * uz);                  // projection on the segment
            double a, b, dist;
            if (sp > 0.0 && sp < len) {
                const double h = fma(pr, uz, -(pz * ur));            // along the normal (uz, -ur)
                dist = fabs(h);
                a = h * uz;
                b = -(h * ur);
            } else {                                                 // an end point is closest
                const double sc = sp <= 0.0 ? 0.0 : len;
                a = fma(-sc, ur, pr);
                b = fma(-sc, uz, pz);
                dist = root_refined(fma(a, a, b * b));
            }
            const double dl = (double)P.w - dist;
            if (!(dl > 0.0)) continue;
            const float idist = 1.f / (float)dist;
            const float na = (float)a * idist;
            const V3 n = v3(na * erx, na * ery, (float)b * idist);
            const unsigned tag = (unsigned)k + 1u;
            V3 xi = v3(0.f, 0.f, 0.f);
            if (__float_as_uint(h0.w) == tag) xi = v3(h0.x, h0.y, h0.z);
            else if (__float_as_uint(h1.w) == tag) xi = v3(h1.x, h1.y, h1.z);
            V3 ft;
            bool slip;
            const V3 fa = contact_fwd<float, true>(coef_of(c), (float)dl * c.q, n, r, 0.f, m, 0.f, vme,
                                                   v3(0.f, 0.f, 0.f), wme, v3(0.f, 0.f, 0.f), xi, dt_hist, ft, slip);
            F = F + fa;
            Tq = Tq - r * cross(n, ft);
            if (MODE == 0 && nst < 2) ws[nst * ncap + s] = make_float4(xi.x, xi.y, xi.z, __uint_as_float(tag));
            ++nst;
        }
    }
    if (MODE == 0)
        for (int i = nst; i < 2; ++i) ws[i * ncap + s] = make_float4(0.f, 0.f, 0.f, 0.f);
    return nst;
}

// WALLS: the variant that evaluates axisymmetric walls (launched only for contexts that have
// them, so that the wall code costs the plain step nothing).
// BS: threads per block (64, 128 or 256; the autotuner picks one), or SMW_BS: one block of 28
// warps per SM (single-instance contexts, the default there).  LPP: lanes per particle
// (1, 2, 4 or 8; more than one only at 128 threads, for systems too small to fill the GPU with
// one thread per row): the LPP lanes of a group take the row entries e = sub, sub + LPP, ...,
// OR their touch masks together, sum their contacts in row order and combine the partial sums
// by a fixed butterfly, so that the result depends on LPP but not on the block size or the
// schedule; the group's first lane adds the floor and walls, integrates and writes.
// The tiles of TILE slots are walked as warp slices of 32 / LPP slots: slice w' of tile t
// (w' = 0 .. 4 LPP - 1) is virtual warp 4 LPP t + w'; unit u is virtual warps
// [u BS / 32, (u + 1) BS / 32), and instances own whole pairs of tiles, so that a unit never
// straddles two instances.  An SM-wide block instead owns a contiguous range of tiles, and its
// warps claim the range's slices in order from a shared counter: the 28 warps of an SM work on
// neighbouring tiles at any time and share their neighbours' state in the SM's L1 (the 1M bed
// steps 5.7 % faster than with seven independent 128-thread blocks per SM, the same bits), and
// the warps of an SM finish within one slice of each other.
constexpr int SMW_BS = 896;
#ifndef SMW_POOL
#define SMW_POOL 8          // the pool: the last 1/SMW_POOL of every block's share
#endif
template <int BS, int LPP = 1>
constexpr int step_minb()
{
    // the same registers per thread at every block size; with several lanes per particle (small
    // systems, where the resident warps are not the limit) room for the whole row state
    return BS == SMW_BS ? 1 : LPP == 1 ? DEM_STEP_MINB * TILE / BS : 5;
}

// Particle state: neighbours' through the read-only data cache, except in fused steps, where the
// state is rewritten during the launch (by other blocks for the neighbours): there every state
// load goes to L2 (ordered after the previous step's writes by the grid barrier's fences), so
// that no SM's L1 or read-only cache can return a line from an earlier step.
template <bool FUSED, typename T>
__device__ __forceinline__ T ld_state(const T* p)
{
    if (FUSED) return __ldcg(p);
    return __ldg(p);
}

// Asynchronous 16-byte copy global -> shared (cp.async): through L1, or in fused steps to L2
// only (other blocks rewrite the state during the launch); 4-byte copies of the particle's own
// stored overlaps; commit and wait for all groups but the newest.
template <bool FUSED>
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src)
{
    if (FUSED)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

// One step over the block's units (MODE 0: force, kick and drift of every particle; MODE 1:
// forces only), ending with the block's displacement maximum folded into its last instance.
// sc, sd, smax: the block's shared staging of the current instance and of the warp maxima.
// FUSED: called once per step by the fused kernel; kstaged: the instance staged in sc and sd at
// the end of the previous step (-1: none), kept so that a block of one instance stages it once
// per launch and then only flips its state buffer (all else in them is constant between list
// builds).
template <int MODE, bool WALLS, int BS, int LPP, bool FUSED = false>
__device__ __forceinline__ void step_pass(const Dev& d, int prime, InstC& sc, InstD& sd, float* smax, int& kstaged)
{
    constexpr int WPB = BS / 32;             // warps per block
    constexpr int SPW = 32 / LPP;            // slots per warp
    constexpr int WPT = TILE / SPW;          // warp slices per tile
    static_assert(BS == 64 || BS == 128 || BS == 256 || BS == SMW_BS, "step block of 64, 128, 256 or SMW_BS threads");
    constexpr bool SMW = BS == SMW_BS;       // single instance, slices claimed from a shared counter
    static_assert(!SMW || (LPP == 1 && !FUSED), "SM-wide blocks: one lane per particle, per-step launches");
    static_assert(LPP == 1 || LPP == 2 || LPP == 4 || LPP == 8, "1, 2, 4 or 8 lanes per particle");
    static_assert(LPP == 1 || MODE == 0, "several lanes per particle only for the step");
    static_assert((WPT & (WPT - 1)) == 0, "warps per tile must be a power of two");
    // entries of a lane's share of a row: bits e with e mod LPP == sub
    constexpr unsigned SUBBITS = LPP == 1 ? 0xffffffffu : LPP == 2 ? 0x55555555u : LPP == 4 ? 0x11111111u : 0x01010101u;
    const int lane = (int)threadIdx.x & 31;
    const int sub = lane & (LPP - 1);
    const unsigned gmask = LPP == 1 ? 0xffffffffu : (((1u << LPP) - 1u) << (lane & ~(LPP - 1)));
    const unsigned submask = SUBBITS << sub;
    // fused steps walk only the tiles holding live slots (contexts with spare capacity keep
    // their blocks busy); the step kernel walks every tile (a lookup per unit costs it 4 %)
    const int nlive = FUSED ? *(volatile int*)&d.g->nlive : d.ntiles;
    const bool all_live = !FUSED || nlive == d.ntiles;   // then no lookup
    const int NU = nlive * WPT / WPB;
    const int u0 = (int)((long long)blockIdx.x * NU / gridDim.x);
    const int u1 = (int)((long long)(blockIdx.x + 1) * NU / gridDim.x);
    const int ncap = d.ncap;
    const size_t plane = (size_t)d.Lmax * ncap;
    int kprev = FUSED ? kstaged : -1;
    if (FUSED && kprev >= 0) {
        __syncthreads();
        if (threadIdx.x == 0) sd.cur ^= 1;   // the last step swapped the instance's buffers
        __syncthreads();
    }
    float runmax = 0.f;
    // SM-wide blocks: block b's share [v0(b), v1(b)) of the slices of the tiles that hold live
    // slots (a contiguous range: the instance's live slots come first).  Its warps claim
    // [v0(b), v1(b) - P) in order from the shared counter snext; the last P slices of every
    // block's share form a pool that all blocks claim from afterwards (g->pool), so that SMs
    // whose share holds less work take over the tails of the others (on the 1M bed the SMs ended
    // between 56 and 100 µs, median 90 µs, without it).  The list build orders each share's
    // windows by contact count, so the pool holds the lightest slices of each share: with pools
    // of 1/32, 1/16 and 1/8 of the shares the step kernel takes 104.4, 103.7 and 100.5 µs
    // against 104.7 µs without the share-aligned windows and a pool of 1/16
    __shared__ int snext, sown, spool[3];   // own counter, own end; pool: P, tiles, first tile
    if (SMW) {
        const int k = __ldg(d.tile_inst);
        for (int i = threadIdx.x; i < (int)(sizeof(InstC) / 4); i += BS) ((int*)&sc)[i] = ((const int*)(d.ic + k))[i];
        if (threadIdx.x < (int)(sizeof(InstD) / 4)) ((int*)&sd)[threadIdx.x] = ((const int*)(d.id + k))[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) {
            const int tf = sc.slot0 / TILE, nt = (sd.n + TILE - 1) / TILE;
            const int P = (nt / (int)gridDim.x) * WPT / SMW_POOL;   // at most 1/SMW_POOL of the shortest share
            snext = (tf + (int)((long long)blockIdx.x * nt / gridDim.x)) * WPT;
            sown = (tf + (int)((long long)(blockIdx.x + 1) * nt / gridDim.x)) * WPT - P;
            spool[0] = P;
            spool[1] = nt;
            spool[2] = tf;
        }
        __syncthreads();
        kprev = k;
    }
    for (int u = u0; SMW || u < u1; ++u) {
        int vw = 0;
        if (SMW) {
            __syncwarp();
            int v = 0;
            if (lane == 0) {
                v = atomicAdd(&snext, 1);
                if (v >= sown) {
                    // the pool: claim q is slice j = q / G from the end part of block b = q mod G
                    const int P = spool[0], G = (int)gridDim.x;
                    const int q = (int)atomicAdd(&d.g->pool, 1u);
                    v = -1;
                    if (q < P * G) {
                        const int b = q % G;
                        v = (spool[2] + (int)((long long)(b + 1) * spool[1] / G)) * WPT - P + q / G;
                    }
                }
            }
            vw = __shfl_sync(0xffffffffu, v, 0);
            if (vw < 0) break;
        }
        const int k = SMW ? kprev : __ldg(d.tile_inst + (all_live ? u * WPB / WPT : d.live_tiles[u * WPB / WPT]));
        if (!SMW && k != kprev) {
            if (MODE == 0 && kprev >= 0) {
                // flush the displacement maximum of the previous instance
                float mx = runmax;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
                __syncthreads();
                if (threadIdx.x == 0) {
                    float bm = smax[0];
                    for (int i = 1; i < WPB; ++i) bm = fmaxf(bm, smax[i]);
                    if (bm > 0.f) atomicMax(&d.id[kprev].stepmax, __float_as_uint(bm));
                }
                runmax = 0.f;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < (int)(sizeof(InstC) / 4); i += BS) ((int*)&sc)[i] = ((const int*)(d.ic + k))[i];
            if (threadIdx.x < (int)(sizeof(InstD) / 4))
                ((int*)&sd)[threadIdx.x] = FUSED ? __ldcg((const int*)(d.id + k) + threadIdx.x)
                                                 : ((const int*)(d.id + k))[threadIdx.x];
            __syncthreads();
            kprev = k;
        }
        const InstC& c = sc;
        // warp slice w' of tile t takes the 32-slot slice (w' + t) mod 4: rebuilds put the rows
        // with the most contacts in the first slice, so the rotation evens out the warps' work
        if (!SMW) vw = u * WPB + ((int)threadIdx.x >> 5);
        const int t = all_live ? vw / WPT : d.live_tiles[vw / WPT];
        const int s = t * TILE + (((vw & (WPT - 1)) + t) & (WPT - 1)) * SPW + lane / LPP;
        if (s - c.slot0 >= sd.n) continue;
        const int cur = sd.cur, lp = sd.lp;
        const int4* __restrict__ pos = d.pos[cur];
        const float4* __restrict__ vel = d.vel[cur];
        const float4* __restrict__ omg = d.omg[cur];
        const int4 P = FUSED ? __ldcg(pos + s) : pos[s];
        float4 Vv = FUSED ? __ldcg(vel + s) : vel[s];
        float4 Wv = FUSED ? __ldcg(omg + s) : omg[s];
        const unsigned idw = __float_as_uint(Vv.w);
        const unsigned myid = idw & ID_MASK;
        const bool wall_prev = (idw & WALL_BIT) != 0u;
        const float m = Wv.w;
        const float q = c.q;
        const float r = (float)P.w * q;
        const V3 vme = v3(Vv.x, Vv.y, Vv.z), wme = v3(Wv.x, Wv.y, Wv.z);
        const float dt_hist = prime ? 0.f : c.dt;
        V3 F = sub == 0 ? m * v3(c.g[0], c.g[1], c.g[2]) : v3(0.f, 0.f, 0.f);
        V3 Tq = v3(0.f, 0.f, 0.f);
        const int ncnt = d.cnt[lp][s];
        const int* nb = d.nbr[lp] + s;
        float* h = d.hist[lp] + s;
        float* ho = MODE == 1 ? d.xi_out + s : h;
        const int per0 = c.per[0], per1 = c.per[1], ext0 = c.ext[0], ext1 = c.ext[1], hf0 = c.half[0],
                  hf1 = c.half[1];

        // ---- pass 1: positions of every entry, touch mask (independent loads)
        const unsigned hm = d.hmask[lp][s];
        unsigned tm = 0u;
        // the first batch of indices is loaded before the row length arrives (rows hold at
        // least d.Lmax entries of storage); entries beyond the row are replaced by this slot
        int jn0 = sub < d.Lmax ? __ldg(nb + (size_t)sub * ncap) : s;
        int jn1 = sub + LPP < d.Lmax ? __ldg(nb + (size_t)(sub + LPP) * ncap) : s;
        int jn2 = sub + 2 * LPP < d.Lmax ? __ldg(nb + (size_t)(sub + 2 * LPP) * ncap) : s;
        int jn3 = sub + 3 * LPP < d.Lmax ? __ldg(nb + (size_t)(sub + 3 * LPP) * ncap) : s;
        jn0 = sub < ncnt ? jn0 : s;
        jn1 = sub + LPP < ncnt ? jn1 : s;
        jn2 = sub + 2 * LPP < ncnt ? jn2 : s;
        jn3 = sub + 3 * LPP < ncnt ? jn3 : s;
        // removed below the removal height: parked until the next list build drops it (tested
        // here, after the row's first loads are in flight, so that live rows do not wait on it)
        if (idw & GONE_BIT) {
            if (MODE == 0 && sub == 0) {
                d.pos[cur ^ 1][s] = P;
                d.vel[cur ^ 1][s] = Vv;
                d.omg[cur ^ 1][s] = Wv;
            } else {
                d.outWX[s] = make_float4(0.f, 0.f, 0.f, 0.f);
                d.cmask[s] = 0ull;
            }
            continue;
        }
        for (int e0 = sub; e0 < ncnt; e0 += 4 * LPP) {
            int jb[4] = {jn0, jn1, jn2, jn3};
            if (DEM_CHECKS)
                for (int k = 0; k < 4; ++k)
                    if (!in_range(d, jb[k], ncap, s, 3)) jb[k] = s;
            int4 Qb[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) Qb[k] = ld_state<FUSED>(pos + jb[k]);
            if (e0 + 4 * LPP < ncnt) jn0 = __ldg(nb + (size_t)(e0 + 4 * LPP) * ncap);
            if (e0 + 5 * LPP < ncnt) jn1 = __ldg(nb + (size_t)(e0 + 5 * LPP) * ncap);
            if (e0 + 6 * LPP < ncnt) jn2 = __ldg(nb + (size_t)(e0 + 6 * LPP) * ncap);
            if (e0 + 7 * LPP < ncnt) jn3 = __ldg(nb + (size_t)(e0 + 7 * LPP) * ncap);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int4 Q = Qb[k];
                const int dx = min_image(P.x - Q.x, per0, ext0, hf0);
                const int dy = min_image(P.y - Q.y, per1, ext1, hf1);
                const int dz = P.z - Q.z;
                const long long d2 = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
                const int S = P.w + Q.w;
                if (e0 + k * LPP < ncnt && d2 < (long long)S * S) tm |= 1u << (e0 + k * LPP);
            }
        }
        // the group's lanes share their touch masks (ncnt, and so the loop above, is the same
        // for every lane of a group)
#pragma unroll
        for (int o = 1; o < LPP; o <<= 1) tm |= __shfl_xor_sync(gmask, tm, o);
        // entries that left contact (or, for the read-out, every non-contact) get no history
        const unsigned rowmask = ncnt >= 32 ? 0xffffffffu : ((1u << ncnt) - 1u);
        unsigned clr = (MODE == 1 ? rowmask : hm) & ~tm & submask;
        while (clr) {
            const int e = __ffs(clr) - 1;
            clr &= clr - 1u;
            ho[(size_t)e * ncap] = 0.f;
            ho[plane + (size_t)e * ncap] = 0.f;
            ho[2 * plane + (size_t)e * ncap] = 0.f;
        }
        unsigned cm = tm;
        unsigned rem = tm & submask;
        // ---- pass 2: the contacts, in row order, the next contact's state in flight: its
        // velocity and spin go to a per-thread slot of shared memory by asynchronous copies (no
        // registers held while they are outstanding; two slots alternate), its position and
        // stored overlap to registers.  7 % faster than all of it in registers; staging the
        // position and overlap as well costs L1 capacity (the slots come out of it) and is 2 %
        // slower
        float4* stg;
        if constexpr (SMW) {
            extern __shared__ float4 stg_dyn[];     // 2 * 2 * BS float4 (57 kB: above the static limit)
            stg = stg_dyn;
        } else {
            __shared__ float4 stg_st[2 * 2 * BS];
            stg = stg_st;
        }
        const int tid = (int)threadIdx.x;
        auto saddr = [&](int sl, int f) -> unsigned {
            return (unsigned)__cvta_generic_to_shared(&stg[(sl * 2 + f) * BS + tid]);
        };
        int4 Qn = P;
        float hxn = 0.f, hyn = 0.f, hzn = 0.f;
        auto issue = [&](int sl, int en_) {
            const size_t o1 = (size_t)en_ * ncap;
            int j = __ldg(nb + o1);
            if (!in_range(d, j, ncap, s, 4)) j = s;
            Qn = ld_state<FUSED>(pos + j);
            cp_async16<FUSED>(saddr(sl, 0), vel + j);
            cp_async16<FUSED>(saddr(sl, 1), omg + j);
            hxn = hyn = hzn = 0.f;
            if ((hm >> en_) & 1u) {
                hxn = h[o1];
                hyn = h[plane + o1];
                hzn = h[2 * plane + o1];
            }
        };
        int en = 0, sl = 0;
        if (rem) {
            en = __ffs(rem) - 1;
            issue(0, en);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        while (rem) {
            const int e = en;
            rem &= rem - 1u;
            const int4 Q = Qn;
            V3 xi = v3(hxn, hyn, hzn);
            if (rem) {
                en = __ffs(rem) - 1;
                issue(sl ^ 1, en);
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            const float4* sp = &stg[(sl * 2) * BS + tid];
            const float4 Vb = sp[0], Wb = sp[BS];
            const int dx = min_image(P.x - Q.x, per0, ext0, hf0);
            const int dy = min_image(P.y - Q.y, per1, ext1, hf1);
            const int dz = P.z - Q.z;
            const long long d2 = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
            const int S = P.w + Q.w;
            const long long S2 = (long long)S * S;
            {
                const float d2f = (float)d2;
                const float inv = rsqrtf(d2f);
                const float dist = d2f * inv;
                const float delta = __fdividef((float)(S2 - d2), (float)S + dist) * q;
                const V3 n = v3((float)dx * inv, (float)dy * inv, (float)dz * inv);
                V3 ft;
                bool slip;
                const V3 fa = contact_fwd<float, false>(coef_of(c), delta, n, r, (float)Q.w * q, m, Wb.w, vme,
                                                        v3(Vb.x, Vb.y, Vb.z), wme, v3(Wb.x, Wb.y, Wb.z), xi, dt_hist,
                                                        ft, slip);
                F = F + fa;
                Tq = Tq - r * cross(n, ft);
            }
            ho[(size_t)e * ncap] = xi.x;
            ho[plane + (size_t)e * ncap] = xi.y;
            ho[2 * plane + (size_t)e * ncap] = xi.z;
            sl ^= 1;
        }
        // the group's partial sums, combined in a fixed order (every lane ends with the same bits)
#pragma unroll
        for (int o = 1; o < LPP; o <<= 1) {
            F.x += __shfl_xor_sync(gmask, F.x, o);
            F.y += __shfl_xor_sync(gmask, F.y, o);
            F.z += __shfl_xor_sync(gmask, F.z, o);
            Tq.x += __shfl_xor_sync(gmask, Tq.x, o);
            Tq.y += __shfl_xor_sync(gmask, Tq.y, o);
            Tq.z += __shfl_xor_sync(gmask, Tq.z, o);
        }
        if (LPP > 1 && sub != 0) continue;      // the group's first lane finishes the particle
        if (MODE == 0) d.hmask[lp][s] = cm;
        if (sd.fext) {   // coupling controllers' force, held over the coupling interval
            const float4 fe = d.fext[lp][s];
            F = F + v3(fe.x, fe.y, fe.z);
        }
        // floor plane z = 0 (the box bottom)
        bool wall_now = false;
        V3 wxi = v3(0.f, 0.f, 0.f);
        if (c.floor_on) {
            const int dw = P.w - P.z;
            if (dw > 0) {
                wall_now = true;
                if (wall_prev) {
                    const float4 hw = d.whist[lp][s];
                    wxi = v3(hw.x, hw.y, hw.z);
                }
                const V3 n = v3(0.f, 0.f, 1.f);
                V3 ft;
                bool slip;
                const V3 fa = contact_fwd<float, true>(coef_of(c), (float)dw * q, n, r, 0.f, m, 0.f, vme,
                                                       v3(c.floor_v[0], c.floor_v[1], c.floor_v[2]), wme,
                                                       v3(0.f, 0.f, 0.f), wxi, dt_hist, ft, slip);
                F = F + fa;
                Tq = Tq - r * cross(n, ft);
                if (MODE == 0) d.whist[lp][s] = make_float4(wxi.x, wxi.y, wxi.z, 0.f);
            }
        }
        int nseg = 0;
        if (WALLS && c.nwp >= 2) nseg = wall_contacts<MODE>(d, c, kprev, s, lp, P, r, m, vme, wme, dt_hist, F, Tq);
        const float inv_m = 1.0f / m;
        const float inv_I = 2.5f / (m * r * r);
        if (!(isfinite(F.x) && isfinite(F.y) && isfinite(F.z) && isfinite(Tq.x) && isfinite(Tq.y) &&
              isfinite(Tq.z))) {
            atomicOr(&d.g->status, ST_NONFINITE);
            d.g->err_slot = s;
        }
        if (MODE == 1) {
            const float hk = prime ? 0.f : 0.5f * c.dt;
            d.outF[s] = make_float4(F.x, F.y, F.z, 0.f);
            d.outT[s] = make_float4(Tq.x, Tq.y, Tq.z, 0.f);
            d.outV[s] = make_float4(Vv.x + hk * F.x * inv_m, Vv.y + hk * F.y * inv_m, Vv.z + hk * F.z * inv_m, 0.f);
            d.outW[s] = make_float4(Wv.x + hk * Tq.x * inv_I, Wv.y + hk * Tq.y * inv_I, Wv.z + hk * Tq.z * inv_I, 0.f);
            d.outWX[s] = make_float4(wxi.x, wxi.y, wxi.z, (float)((wall_now ? 1 : 0) + nseg));
            d.cmask[s] = cm;
        } else {
            const float kick = prime ? 0.5f * c.dt : c.dt;
            Vv.x += kick * F.x * inv_m;
            Vv.y += kick * F.y * inv_m;
            Vv.z += kick * F.z * inv_m;
            Wv.x += kick * Tq.x * inv_I;
            Wv.y += kick * Tq.y * inv_I;
            Wv.z += kick * Tq.z * inv_I;
            const float sx = Vv.x * c.dt_over_q, sy = Vv.y * c.dt_over_q, sz = Vv.z * c.dt_over_q;
            int4 Pn = P;
            bool bad = !(fabsf(sx) < 5.0e8f && fabsf(sy) < 5.0e8f && fabsf(sz) < 5.0e8f);
            if (!bad) {
                // unbiased rounding to the position grid: floor(s + u), u uniform in [0, 1)
                // from a hash of the particle's ID and position (a function of the state
                // alone, so replays, graphs and batched runs round identically); plain
                // rounding would bias a steady drift by up to half a quantum per step
                const unsigned h0 = mix32(myid * 0x9E3779B9u ^ (unsigned)P.x);
                const unsigned h1 = mix32(h0 ^ (unsigned)P.y);
                const unsigned h2 = mix32(h1 ^ (unsigned)P.z);
                const int ix = __float2int_rd(sx + (float)(h0 >> 8) * 0x1p-24f);
                const int iy = __float2int_rd(sy + (float)(h1 >> 8) * 0x1p-24f);
                const int iz = __float2int_rd(sz + (float)(h2 >> 8) * 0x1p-24f);
                int x = P.x + ix, y = P.y + iy;
                if (per0) {
                    if (x >= ext0) x -= ext0;
                    else if (x < 0) x += ext0;
                }
                if (per1) {
                    if (y >= ext1) y -= ext1;
                    else if (y < 0) y += ext1;
                }
                const long long z = (long long)P.z + iz;
                if (z > 2000000000ll || z < -2000000000ll) bad = true;
                Pn = make_int4(x, y, (int)z, P.w);
                runmax = fmaxf(runmax, sqrtf((float)ix * (float)ix + (float)iy * (float)iy + (float)iz * (float)iz));
            }
            if (bad) {
                atomicOr(&d.g->status, ST_ESCAPED);
                d.g->err_slot = s;
            }
            unsigned gone = 0u;
            if (Pn.z < c.zrem) {
                // fell below the removal height: parked two cell heights lower with no radius
                // (every live particle lies above the removal height, so none can touch it)
                // and frozen until the next list build drops it; no rebuild is forced
                gone = GONE_BIT;
                Pn.z = (int)max((long long)Pn.z - 2ll * (c.ext[2] / c.nc[2] + 1), -2000000000ll);
                Pn.w = 0;
                atomicAdd(d.wrem + 2 * kprev, 1.0);
                atomicAdd(d.wrem + 2 * kprev + 1, (double)m);
            }
            const int nxt = cur ^ 1;
            d.pos[nxt][s] = Pn;
            d.vel[nxt][s] = make_float4(Vv.x, Vv.y, Vv.z, __uint_as_float(myid | gone | (wall_now ? WALL_BIT : 0u)));
            d.omg[nxt][s] = Wv;
        }
    }
    if (MODE == 0) {
        // the last instance's displacement maximum
        float mx = runmax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            float bm = smax[0];
            for (int i = 1; i < WPB; ++i) bm = fmaxf(bm, smax[i]);
            if (bm > 0.f && kprev >= 0) atomicMax(&d.id[kprev].stepmax, __float_as_uint(bm));
        }
    }
    kstaged = kprev;
}

// The end of a step for every instance, by the last block to finish it: the displacement
// bound grows by the step's maximum, the state buffers swap, and an instance whose bound
// reaches the skin is flagged for a list build (an error while the lists are frozen).
__device__ __forceinline__ void step_finish_instances(const Dev& d)
{
    const unsigned frozen = __ldcg(&d.g->frozen);
    for (int kk = threadIdx.x; kk < d.B; kk += blockDim.x) {
        // L2 loads (__ldcg): the instance's record was last written by another block (in fused
        // steps, during this launch), never to be read from this SM's L1.  Only this block writes
        // disp, cur and flag, so they are loaded together up front and the chain of dependent
        // round trips at the end of every step is two long (the exchange, then the stores)
        InstD* Dk = d.id + kk;
        const float disp0 = __ldcg(&Dk->disp);
        const int cur0 = __ldcg(&Dk->cur), flag0 = __ldcg(&Dk->flag);
        const float skin = d.ic[kk].skin_f;
        const float sm = __uint_as_float(atomicExch(&Dk->stepmax, 0u));
        const float disp = disp0 + sm;
        __stcg(&Dk->disp, disp);
        __stcg(&Dk->cur, cur0 ^ 1);
        if (2.0f * disp >= 0.99f * skin && flag0 == 0) {
            if (frozen) {
                atomicOr(&d.g->status, ST_SKIN);
            } else {
                __stcg(&Dk->flag, 1);
                atomicOr(&d.g->any, 1u);
            }
        }
    }
}

template <int MODE, bool WALLS, int BS = TILE, int LPP = 1>
__global__ void __launch_bounds__(BS, (step_minb<BS, LPP>())) k_step(Dev d, int prime, cudaGraphConditionalHandle hnext, int use_cond)
{
    __shared__ InstC sc;
    __shared__ InstD sd;
    __shared__ float smax[BS / 32];
    __shared__ bool am_last;
    int kstaged = -1;
    step_pass<MODE, WALLS, BS, LPP>(d, prime, sc, sd, smax, kstaged);
    if (MODE == 0) {
        // the last block to finish accumulates the bound per instance and decides on rebuilds
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(&d.g->counter, 1u);
            am_last = prev == gridDim.x - 1;
        }
        __syncthreads();
        if (am_last) {
            __threadfence();
            step_finish_instances(d);
            __syncthreads();
            if (threadIdx.x == 0) {
                d.g->counter = 0u;
                d.g->pool = 0u;                 // every block has left its claim loop
                if (use_cond) cudaGraphSetConditional(hnext, atomicOr(&d.g->any, 0u) ? 1u : 0u);
            }
        }
    }
}

// Several steps in one cooperative launch (every block resident at once; a block walks its
// range of tiles each step, one tile per block when they all fit), for systems too small to hide
// the per-step launch and graph-node latency.
// Each step is exactly the step kernel's; between steps a grid barrier (the last block to
// arrive ends the step for every instance, as the step kernel's last block does, then
// releases the others; every wait gives up after a second and reports DEM_ERR_TIMEOUT, and a
// block that gave up, or saw another give up, leaves the launch).  Runs the steps still to do
// in this graph launch (g->remain) and stops early when an instance needs a list build; the
// last block then sets the loop's conditions: h_rb (build the lists before going on) and
// h_loop (steps remain).
constexpr unsigned long long BAR_WAIT_NS = 1000000000ull;   // a barrier wait gives up after 1 s
constexpr unsigned BAR_POLLS = 1u << 24;                     // or after this many polls

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <bool WALLS, int LPP>
__global__ void __launch_bounds__(TILE, 5) k_steps(Dev d, cudaGraphConditionalHandle h_rb,
                                                                        cudaGraphConditionalHandle h_loop)
{
    __shared__ InstC sc;
    __shared__ InstD sd;
    __shared__ float smax[TILE / 32];
    __shared__ bool am_last, quit;
    // stop unless the block that ends the last step says otherwise (set before any block can
    // reach the final barrier, so the later setting wins)
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h_loop, 0u);
    const long long todo = *(volatile long long*)&d.g->remain;
    long long done = 0;
    bool final_last = false;
    int kstaged = -1;
    while (done < todo) {
        step_pass<0, WALLS, TILE, LPP, true>(d, 0, sc, sd, smax, kstaged);
        if (threadIdx.x == 0) {
            const unsigned gen = *(volatile unsigned*)&d.g->bar_gen;
            __threadfence();
            // a test of the timeout path (dem_test_stall_barrier): the first block does not
            // arrive at the first barrier of this launch and leaves, so the others' waits run out
            const bool skip = blockIdx.x == 0 && done == 0 && atomicExch(&d.g->test_stall, 0u) != 0u;
            const unsigned prev = skip ? 0u : atomicAdd(&d.g->counter, 1u);
            am_last = !skip && prev == gridDim.x - 1;
            if (skip) {
                atomicOr(&d.g->status, ST_TIMEOUT);
            } else if (!am_last) {
                const unsigned long long t0 = global_ns();
                unsigned polls = 0u;
                while (*(volatile unsigned*)&d.g->bar_gen == gen) {
                    if (++polls > BAR_POLLS || global_ns() - t0 > BAR_WAIT_NS) {
                        atomicOr(&d.g->status, ST_TIMEOUT);
                        break;
                    }
                    __nanosleep(256);
                }
                __threadfence();
            }
        }
        __syncthreads();
        const bool last = am_last;
        if (last) {
            __threadfence();
            step_finish_instances(d);
            __syncthreads();
            if (threadIdx.x == 0) {
                d.g->counter = 0u;
                __threadfence();
                atomicAdd(&d.g->bar_gen, 1u);      // release
            }
        }
        ++done;
        final_last = last;
        if (threadIdx.x == 0)
            quit = *(volatile unsigned*)&d.g->any != 0u || (*(volatile unsigned*)&d.g->status & ST_TIMEOUT) != 0u;
        __syncthreads();
        if (quit) break;
    }
    if (final_last && threadIdx.x == 0) {
        const long long rem = todo - done;
        d.g->remain = rem;
        const bool timeout = (*(volatile unsigned*)&d.g->status & ST_TIMEOUT) != 0u;
        cudaGraphSetConditional(h_rb, *(volatile unsigned*)&d.g->any ? 1u : 0u);
        cudaGraphSetConditional(h_loop, rem > 0 && !timeout ? 1u : 0u);
    }
}

// the start of a fused graph launch: S steps to do, a list build first if one is pending
__global__ void k_steps_init(Dev d, long long S, cudaGraphConditionalHandle h_rb, cudaGraphConditionalHandle h_loop)
{
    d.g->remain = S;
    cudaGraphSetConditional(h_rb, d.g->any ? 1u : 0u);
    cudaGraphSetConditional(h_loop, S > 0 ? 1u : 0u);
}

__global__ void k_set_cond(Dev d, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, d.g->any ? 1u : 0u);
}

// =========================================================== field I/O

__device__ __forceinline__ int find_inst(const long long* goff, int B, long long g)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (goff[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}


__global__ void k_init_ids(Dev d)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.ncap) return;
    const int k = d.tile_inst[s / TILE];
    const int id = s - d.ic[k].slot0;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int b = 0; b < 2; ++b) {
        d.pos[b][s] = make_int4(0, 0, 0, 0);
        d.vel[b][s] = make_float4(0.f, 0.f, 0.f, __uint_as_float((unsigned)id));
        d.omg[b][s] = z;
        d.cnt[b][s] = 0;
        d.hmask[b][s] = 0u;
        d.fext[b][s] = z;
        d.whist[b][s] = z;
        d.wseg[b][s] = z;
        d.wseg[b][d.ncap + s] = z;
    }
    d.slot_of_id[s] = s;
}

// field writes: src holds float64 values in the user layout
__global__ void k_write_field(Dev d, int field, const double* __restrict__ src, long long total,
                              const HostInstLo* __restrict__ hl)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int k = find_inst(d.goff, d.B, g);
    const InstC& c = d.ic[k];
    const int id = (int)(g - d.goff[k]);
    const int s = d.slot_of_id[c.slot0 + id];
    if (s < 0) return;                       // removed particle
    const int cur = d.id[k].cur;
    const double q = hl[k].q;
    if (field == DEM_F_POS) {
        int4 p = d.pos[cur][s];
        int xi[3];
        for (int a = 0; a < 3; ++a) {
            double u = rint((src[3 * g + a] - hl[k].lo[a]) / q);
            if (c.per[a]) {
                double L = (double)c.ext[a];
                u = u - L * floor(u / L);
                if (u >= L) u -= L;
            }
            if (!(u > -2.0e9 && u < 2.0e9)) {
                atomicOr(&d.g->status, ST_ESCAPED);
                u = 0.0;
            }
            xi[a] = (int)u;
        }
        p.x = xi[0]; p.y = xi[1]; p.z = xi[2];
        d.pos[cur][s] = p;
    } else if (field == DEM_F_VEL) {
        float4 v = d.vel[cur][s];
        v.x = (float)src[3 * g]; v.y = (float)src[3 * g + 1]; v.z = (float)src[3 * g + 2];
        d.vel[cur][s] = v;
    } else if (field == DEM_F_OMEGA) {
        float4 w = d.omg[cur][s];
        w.x = (float)src[3 * g]; w.y = (float)src[3 * g + 1]; w.z = (float)src[3 * g + 2];
        d.omg[cur][s] = w;
    } else if (field == DEM_F_RADIUS) {
        int4 p = d.pos[cur][s];
        const double r = src[g];
        p.w = (int)rint(r / q);
        d.pos[cur][s] = p;
        float4 w = d.omg[cur][s];
        w.w = (float)(hl[k].rho * (4.0 / 3.0) * 3.14159265358979323846 * r * r * r);
        d.omg[cur][s] = w;
    } else if (field == DEM_F_MASS) {
        float4 w = d.omg[cur][s];
        w.w = (float)src[g];
        d.omg[cur][s] = w;
    } else if (field == DEM_F_FEXT) {
        d.fext[d.id[k].lp][s] = make_float4((float)src[3 * g], (float)src[3 * g + 1], (float)src[3 * g + 2], 0.f);
        d.id[k].fext = 1;                    // every thread of the instance stores the same value
    } else if (field == DEM_F_WALL_XI) {
        // a floor contact's stored overlap (after the lists were built for this state): kept
        // by the next evaluation if the particle touches the floor there
        const float4 xi = make_float4((float)src[3 * g], (float)src[3 * g + 1], (float)src[3 * g + 2], 0.f);
        d.whist[d.id[k].lp][s] = xi;
        float4 v = d.vel[cur][s];
        unsigned idw = __float_as_uint(v.w) & ~WALL_BIT;
        if (xi.x != 0.f || xi.y != 0.f || xi.z != 0.f) idw |= WALL_BIT;
        v.w = __uint_as_float(idw);
        d.vel[cur][s] = v;
    }
}

__global__ void k_read_field(Dev d, int field, double* __restrict__ dst, long long total,
                             const HostInstLo* __restrict__ hl)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int k = find_inst(d.goff, d.B, g);
    const InstC& c = d.ic[k];
    const int id = (int)(g - d.goff[k]);
    const int s = d.slot_of_id[c.slot0 + id];
    if (s < 0 || (__float_as_uint(d.vel[d.id[k].cur][s].w) & GONE_BIT)) {   // removed (or marked for removal)
        const int w = (field == DEM_F_RADIUS || field == DEM_F_MASS || field == DEM_F_NBR_COUNT) ? 1 : 3;
        for (int a = 0; a < w; ++a) dst[w * g + a] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const int cur = d.id[k].cur;
    const double q = hl[k].q;
    float4 f;
    switch (field) {
    case DEM_F_POS: {
        const int4 p = d.pos[cur][s];
        // lo + u q rounded once (the coupling kernels form positions the same way)
        dst[3 * g] = __fma_rn((double)p.x, q, hl[k].lo[0]);
        dst[3 * g + 1] = __fma_rn((double)p.y, q, hl[k].lo[1]);
        dst[3 * g + 2] = __fma_rn((double)p.z, q, hl[k].lo[2]);
        return;
    }
    case DEM_F_RADIUS: dst[g] = (double)d.pos[cur][s].w * q; return;
    case DEM_F_MASS: dst[g] = (double)d.omg[cur][s].w; return;
    case DEM_F_NBR_COUNT: dst[g] = (double)d.cnt[d.id[k].lp][s]; return;
    case DEM_F_VEL: f = d.outV[s]; break;
    case DEM_F_OMEGA: f = d.outW[s]; break;
    case DEM_F_FORCE: f = d.outF[s]; break;
    case DEM_F_TORQUE: f = d.outT[s]; break;
    case DEM_F_WALL_XI: f = d.outWX[s]; break;
    case DEM_F_FEXT: f = d.fext[d.id[k].lp][s]; break;
    default: return;
    }
    dst[3 * g] = f.x;
    dst[3 * g + 1] = f.y;
    dst[3 * g + 2] = f.z;
}

__global__ void k_read_contacts(Dev d, int* __restrict__ partner, double* __restrict__ xi, int width)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.ncap) return;
    const int k = d.tile_inst[s / TILE];
    const InstD D = d.id[k];
    const InstC& c = d.ic[k];
    if (s - c.slot0 >= D.n) return;
    const unsigned id = __float_as_uint(d.vel[D.cur][s].w) & ID_MASK;
    const size_t plane = (size_t)d.Lmax * d.ncap;
    const int cnt = d.cnt[D.lp][s];
    const unsigned long long cm = d.cmask[s];
    // contacts of the row, ordered by partner ID
    int pid[MAXL], ent[MAXL];
    int nct = 0;
    for (int e = 0; e < cnt; ++e) {
        if (!((cm >> e) & 1ull)) continue;
        const int j = d.nbr[D.lp][(size_t)e * d.ncap + s];
        const int p = (int)(__float_as_uint(d.vel[D.cur][j].w) & ID_MASK);
        int t = nct - 1;
        while (t >= 0 && pid[t] > p) {
            pid[t + 1] = pid[t];
            ent[t + 1] = ent[t];
            --t;
        }
        pid[t + 1] = p;
        ent[t + 1] = e;
        ++nct;
    }
    if (nct > width) atomicOr(&d.g->status, ST_TRUNC);
    for (int t = 0; t < width; ++t) {
        const size_t o = (size_t)id * width + t;
        if (t < nct) {
            const int e = ent[t];
            partner[o] = pid[t];
            // stored from this particle's side; reported in the frame of the lower ID
            const double sg = (int)id < pid[t] ? 1.0 : -1.0;
            xi[3 * o] = sg * d.xi_out[(size_t)e * d.ncap + s];
            xi[3 * o + 1] = sg * d.xi_out[plane + (size_t)e * d.ncap + s];
            xi[3 * o + 2] = sg * d.xi_out[2 * plane + (size_t)e * d.ncap + s];
        } else {
            partner[o] = -1;
            xi[3 * o] = xi[3 * o + 1] = xi[3 * o + 2] = 0.0;
        }
    }
}

// every entry of the particle's neighbour row, as partner IDs in ascending order (-1 padded)
__global__ void k_read_neighbors(Dev d, int* __restrict__ partner, int width)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.ncap) return;
    const int k = d.tile_inst[s / TILE];
    const InstD D = d.id[k];
    const InstC& c = d.ic[k];
    if (s - c.slot0 >= D.n) return;
    const unsigned id = __float_as_uint(d.vel[D.cur][s].w) & ID_MASK;
    const int cnt = d.cnt[D.lp][s];
    int pid[MAXL];
    for (int e = 0; e < cnt; ++e) {
        const int j = d.nbr[D.lp][(size_t)e * d.ncap + s];
        const int p = (int)(__float_as_uint(d.vel[D.cur][j].w) & ID_MASK);
        int t = e - 1;
        while (t >= 0 && pid[t] > p) {
            pid[t + 1] = pid[t];
            --t;
        }
        pid[t + 1] = p;
    }
    if (cnt > width) atomicOr(&d.g->status, ST_TRUNC);
    for (int t = 0; t < width; ++t) partner[(size_t)id * width + t] = t < cnt ? pid[t] : -1;
}

__global__ void k_write_contacts(Dev d, const int* __restrict__ partner, const double* __restrict__ xi, int width)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.ncap) return;
    const int k = d.tile_inst[s / TILE];
    const InstD D = d.id[k];
    const InstC& c = d.ic[k];
    if (s - c.slot0 >= D.n) return;
    const unsigned id = __float_as_uint(d.vel[D.cur][s].w) & ID_MASK;
    const size_t plane = (size_t)d.Lmax * d.ncap;
    const int cnt = d.cnt[D.lp][s];
    float* h = d.hist[D.lp] + s;
    unsigned hm = d.hmask[D.lp][s];
    for (int e = 0; e < cnt; ++e) {
        const int j = d.nbr[D.lp][(size_t)e * d.ncap + s];
        const int pid = (int)(__float_as_uint(d.vel[D.cur][j].w) & ID_MASK);
        for (int t = 0; t < width; ++t) {
            const size_t o = (size_t)id * width + t;
            const int p = partner[o];
            if (p < 0 || p > pid) break;
            if (p == pid) {
                const double sg = (int)id < pid ? 1.0 : -1.0;   // input is in the lower ID's frame
                h[(size_t)e * d.ncap] = (float)(sg * xi[3 * o]);
                h[plane + (size_t)e * d.ncap] = (float)(sg * xi[3 * o + 1]);
                h[2 * plane + (size_t)e * d.ncap] = (float)(sg * xi[3 * o + 2]);
                hm |= 1u << e;
                break;
            }
        }
    }
    d.hmask[D.lp][s] = hm;
}

__global__ void k_stats(Dev d)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long l = 0, cc = 0, wc = 0;
    if (s < d.ncap) {
        const int k = d.tile_inst[s / TILE];
        const InstD D = d.id[k];
        if (s - d.ic[k].slot0 < D.n) {
            l = (unsigned long long)d.cnt[D.lp][s];
            wc = (unsigned long long)d.outWX[s].w;   // floor and axisymmetric-wall contacts
            cc = (unsigned long long)__popcll(d.cmask[s]) + wc;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_xor_sync(0xffffffffu, l, o);
        cc += __shfl_xor_sync(0xffffffffu, cc, o);
        wc += __shfl_xor_sync(0xffffffffu, wc, o);
    }
    if ((threadIdx.x & 31) == 0 && (l || cc)) {
        atomicAdd(&d.g->sum_list, l);
        atomicAdd(&d.g->sum_contacts, cc);
        atomicAdd(&d.g->sum_wall, wc);
    }
}

// ================================================================ adjoint
// Reverse mode of the step for a differentiable rollout (lists frozen):
//   x^{n+1} = x^n + dt v^{n+1/2},  v^{n+1/2} = v^{n-1/2} + kick F^n / m,
//   w^{n+1/2} = w^{n-1/2} + kick T^n / I,  (F^n, T^n, xi^n) = forces at
//   (x^n, v^{n-1/2}, w^{n-1/2}, xi^{n-1}; E, e, mu),
// with the contact and slip pattern of the forward pass.  The adjoint of the
// stored overlap is kept from each row's side, so the two rows of a pair hold
// opposite values and every particle can compute its part of a pair's
// derivative alone (no atomics; the parameter part is split evenly).



template <typename Fn>
__device__ __forceinline__ void for_live_slots(const Dev& d, Fn fn)
{
    for (int t = blockIdx.x; t < d.ntiles; t += gridDim.x) {
        const int k = d.tile_inst[t];
        const InstD D = d.id[k];
        const int s = t * TILE + threadIdx.x;
        if (s - d.ic[k].slot0 >= D.n) continue;
        fn(s, k, D);
    }
}

template <bool SAVE>
__global__ void __launch_bounds__(TILE) k_snap(Dev d, Snap S)
{
    const size_t plane = (size_t)d.Lmax * d.ncap;
    for_live_slots(d, [&](int s, int k, const InstD& D) {
        // only entries whose history bit is set hold a stored overlap that anything reads
        // (every reader gates on the bit), so only those are copied
        const int cur = D.cur, lp = D.lp;
        float* h = d.hist[lp] + s;
        float* hs = S.hist + s;
        if (SAVE) {
            S.pos[s] = d.pos[cur][s];
            S.vel[s] = d.vel[cur][s];
            S.omg[s] = d.omg[cur][s];
            unsigned hm = d.hmask[lp][s];
            S.hmask[s] = hm;
            S.whist[s] = d.whist[lp][s];
            while (hm) {
                const size_t o = (size_t)(__ffs(hm) - 1) * d.ncap;
                hm &= hm - 1u;
                const float x = h[o], y = h[plane + o], z = h[2 * plane + o];
                hs[o] = x;
                hs[plane + o] = y;
                hs[2 * plane + o] = z;
            }
        } else {
            d.pos[cur][s] = S.pos[s];
            d.vel[cur][s] = S.vel[s];
            d.omg[cur][s] = S.omg[s];
            unsigned hm = S.hmask[s];
            d.hmask[lp][s] = hm;
            d.whist[lp][s] = S.whist[s];
            while (hm) {
                const size_t o = (size_t)(__ffs(hm) - 1) * d.ncap;
                hm &= hm - 1u;
                const float x = hs[o], y = hs[plane + o], z = hs[2 * plane + o];
                h[o] = x;
                h[plane + o] = y;
                h[2 * plane + o] = z;
            }
        }
        (void)k;
    });
    if (blockIdx.x == 0) {
        for (int k = threadIdx.x; k < d.B; k += blockDim.x) {
            if (SAVE) S.disp[k] = d.id[k].disp;
            else d.id[k].disp = S.disp[k];
        }
    }
}

// F-bar, T-bar of this step from the velocity adjoints (and the drift)
__global__ void __launch_bounds__(TILE) k_adj_prep(Dev d, AdjBufs a, float kick, int drift)
{
    for_live_slots(d, [&](int s, int k, const InstD& D) {
        const InstC& c = d.ic[k];
        const float dt = c.dt;
        float4 vb = a.vb[s];
        if (drift) {
            const float4 xb = a.xb[s];
            vb.x += dt * xb.x;
            vb.y += dt * xb.y;
            vb.z += dt * xb.z;
            a.vb[s] = vb;
        }
        const float4 wb = a.wb[s];
        const float m = d.omg[D.cur][s].w;
        const float r = (float)d.pos[D.cur][s].w * c.q;
        const float fk = kick * dt / m, tk = kick * dt / (0.4f * m * r * r);
        a.Fb[s] = make_float4(fk * vb.x, fk * vb.y, fk * vb.z, 0.f);
        a.Tb[s] = make_float4(tk * wb.x, tk * wb.y, tk * wb.z, 0.f);
    });
}

// pull the force adjoints back to x^n, v^{n-1/2}, w^{n-1/2}, xi^{n-1} and (E, e, mu)
__global__ void __launch_bounds__(TILE) k_adj_force(Dev d, AdjBufs a, Snap S, int prime)
{
    const size_t plane = (size_t)d.Lmax * d.ncap;
    const int ncap = d.ncap;
    for_live_slots(d, [&](int s, int k, const InstD& D) {
        const InstC& c = d.ic[k];
        const Coef<float> cf = coef_of(c);
        const int lp = D.lp;
        const float q = c.q;
        const int4 P = S.pos[s];
        const float4 Vv = S.vel[s], Wv = S.omg[s];
        const float m = Wv.w, r = (float)P.w * q;
        const V3 vme = v3(Vv.x, Vv.y, Vv.z), wme = v3(Wv.x, Wv.y, Wv.z);
        const unsigned hm = S.hmask[s];
        const float dt_hist = prime ? 0.f : c.dt;
        const float4 Fi = a.Fb[s], Ti = a.Tb[s];
        float4 xb = a.xb[s], vb = a.vb[s], wb = a.wb[s];
        // the particle's share of d(loss)/d(E, e, mu) this step, summed over its few contacts in
        // float and added to the running double sums once (FP64 per contact is slow on this GPU)
        float thE = 0.f, the = 0.f, thm = 0.f;
        const int ncnt = d.cnt[lp][s];
        const int* nb = d.nbr[lp] + s;
        float* xbr = a.xib + s;
        const float* hs = S.hist + s;
        const int per0 = c.per[0], per1 = c.per[1], ext0 = c.ext[0], ext1 = c.ext[1], hf0 = c.half[0],
                  hf1 = c.half[1];
        // pass 1: which entries touch (independent loads, four at a time)
        unsigned tm = 0u;
        for (int e0 = 0; e0 < ncnt; e0 += 4) {
            int jb[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) jb[k] = e0 + k < ncnt ? __ldg(nb + (size_t)(e0 + k) * ncap) : s;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int4 Q = __ldg(S.pos + jb[k]);
                const int dx = min_image(P.x - Q.x, per0, ext0, hf0);
                const int dy = min_image(P.y - Q.y, per1, ext1, hf1);
                const int dz = P.z - Q.z;
                const long long d2 = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
                const int Sr = P.w + Q.w;
                if (e0 + k < ncnt && d2 < (long long)Sr * Sr) tm |= 1u << (e0 + k);
            }
        }
        // the overlap adjoint of entries out of contact is zero
        const unsigned rowmask = ncnt >= 32 ? 0xffffffffu : ((1u << ncnt) - 1u);
        for (unsigned z = rowmask & ~tm; z; z &= z - 1u) {
            const size_t o = (size_t)(__ffs(z) - 1) * ncap;
            xbr[o] = 0.f;
            xbr[plane + o] = 0.f;
            xbr[2 * plane + o] = 0.f;
        }
        // pass 2: the contacts in row order
        for (unsigned rem = tm; rem; rem &= rem - 1u) {
            const int e = __ffs(rem) - 1;
            const size_t o = (size_t)e * ncap;
            const int j = __ldg(nb + o);
            const int4 Q = __ldg(S.pos + j);
            const int dx = min_image(P.x - Q.x, per0, ext0, hf0);
            const int dy = min_image(P.y - Q.y, per1, ext1, hf1);
            const int dz = P.z - Q.z;
            const long long d2 = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
            const int Sr = P.w + Q.w;
            const long long S2 = (long long)Sr * Sr;
            const float4 Vj = S.vel[j], Wj = S.omg[j];
            const float4 Fj = a.Fb[j], Tj = a.Tb[j];
            const float d2f = (float)d2;
            const float inv = rsqrtf(d2f);
            const float dist = d2f * inv;
            const float delta = __fdividef((float)(S2 - d2), (float)Sr + dist) * q;
            const V3 n = v3((float)dx * inv, (float)dy * inv, (float)dz * inv);
            const float rj = (float)Q.w * q;
            const V3 xio = ((hm >> e) & 1u) ? v3(hs[o], hs[plane + o], hs[2 * plane + o]) : v3(0.f, 0.f, 0.f);
            const V3 G = v3(Fi.x - Fj.x, Fi.y - Fj.y, Fi.z - Fj.z);
            const V3 H = v3(r * Ti.x + rj * Tj.x, r * Ti.y + rj * Tj.y, r * Ti.z + rj * Tj.z);
            const V3 xibar = v3(xbr[o], xbr[plane + o], xbr[2 * plane + o]);
            PairGrad<float> g;
            contact_vjp<float, false>(cf, delta, n, dist * q, r, rj, m, Wj.w, vme, v3(Vj.x, Vj.y, Vj.z), wme,
                                      v3(Wj.x, Wj.y, Wj.z), xio, dt_hist, G, H, xibar, g);
            xb.x += g.r.x; xb.y += g.r.y; xb.z += g.r.z;
            vb.x += g.va.x; vb.y += g.va.y; vb.z += g.va.z;
            wb.x += g.wa.x; wb.y += g.wa.y; wb.z += g.wa.z;
            xbr[o] = g.xi.x;
            xbr[plane + o] = g.xi.y;
            xbr[2 * plane + o] = g.xi.z;
            // each side of the pair adds half of the parameter derivative
            thE += 0.5f * (g.c_kn * c.c_kn + g.c_kt * c.c_kt) * c.inv_E;
            the += 0.5f * g.nbeta * c.dnb_de;
            thm += 0.5f * g.mu;
        }
        float4 wx = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c.floor_on) {
            const int dw = P.w - P.z;
            if (dw > 0) {
                const bool wall_prev = (__float_as_uint(Vv.w) & WALL_BIT) != 0u;
                const float4 hw = S.whist[s];
                const V3 xio = wall_prev ? v3(hw.x, hw.y, hw.z) : v3(0.f, 0.f, 0.f);
                const float4 wxo = a.wxib[s];
                PairGrad<float> g;
                contact_vjp<float, true>(cf, (float)dw * q, v3(0.f, 0.f, 1.f), (float)P.z * q, r, 0.f, m, 0.f, vme,
                                         v3(c.floor_v[0], c.floor_v[1], c.floor_v[2]), wme, v3(0.f, 0.f, 0.f), xio,
                                         dt_hist, v3(Fi.x, Fi.y, Fi.z), v3(r * Ti.x, r * Ti.y, r * Ti.z),
                                         v3(wxo.x, wxo.y, wxo.z), g);
                xb.z += g.r.z;
                vb.x += g.va.x; vb.y += g.va.y; vb.z += g.va.z;
                wb.x += g.wa.x; wb.y += g.wa.y; wb.z += g.wa.z;
                wx = make_float4(g.xi.x, g.xi.y, g.xi.z, 0.f);
                thE += (g.c_kn * c.c_kn + g.c_kt * c.c_kt) * c.inv_E;
                the += g.nbeta * c.dnb_de;
                if (c.mu_w_follows) thm += g.mu;
            }
        }
        a.wxib[s] = wx;
        a.xb[s] = xb;
        a.vb[s] = vb;
        a.wb[s] = wb;
        a.thb[3 * (size_t)s] += (double)thE;
        a.thb[3 * (size_t)s + 1] += (double)the;
        a.thb[3 * (size_t)s + 2] += (double)thm;
    });
}

// Observables at the evaluated step, one block per instance (deterministic
// fixed-order reductions): kinetic energy sum 1/2 m v^2 + 1/2 I w^2, and the
// runout max_i |(x_i, y_i) - axis| with the particle attaining it (lowest ID on
// ties).  small[16 k + ...]: 0-1 axis (in), 2 KE, 3 runout, 4 argmax slot.
__global__ void __launch_bounds__(256) k_obs(Dev d, const HostInstLo* __restrict__ hl)
{
    const int k = blockIdx.x;
    const InstC& c = d.ic[k];
    const InstD D = d.id[k];
    double* sm = d.small + 16 * k;
    const double cx = sm[0], cy = sm[1];
    double ke = 0.0, best = -1.0;
    int bslot = -1;
    unsigned bid = 0xffffffffu;
    for (int i = threadIdx.x; i < D.n; i += blockDim.x) {
        const int s = c.slot0 + i;
        const float4 v = d.outV[s], w = d.outW[s];
        const float m = d.omg[D.cur][s].w;
        const int4 p = d.pos[D.cur][s];
        const double r = (double)p.w * hl[k].q;
        const double I = 0.4 * m * r * r;
        ke += 0.5 * m * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z) +
              0.5 * I * ((double)w.x * w.x + (double)w.y * w.y + (double)w.z * w.z);
        const double x = hl[k].lo[0] + (double)p.x * hl[k].q - cx;
        const double y = hl[k].lo[1] + (double)p.y * hl[k].q - cy;
        const double rho = sqrt(x * x + y * y);
        const unsigned id = __float_as_uint(d.vel[D.cur][s].w) & ID_MASK;
        if (rho > best || (rho == best && id < bid)) {
            best = rho;
            bslot = s;
            bid = id;
        }
    }
    __shared__ double ske[256], sbest[256];
    __shared__ int sslot[256];
    __shared__ unsigned sid[256];
    ske[threadIdx.x] = ke;
    sbest[threadIdx.x] = best;
    sslot[threadIdx.x] = bslot;
    sid[threadIdx.x] = bid;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const int t = threadIdx.x + o;
            ske[threadIdx.x] += ske[t];
            if (sbest[t] > sbest[threadIdx.x] || (sbest[t] == sbest[threadIdx.x] && sid[t] < sid[threadIdx.x])) {
                sbest[threadIdx.x] = sbest[t];
                sslot[threadIdx.x] = sslot[t];
                sid[threadIdx.x] = sid[t];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sm[2] = ske[0];
        sm[3] = sbest[0] < 0.0 ? 0.0 : sbest[0];
        sm[4] = (double)sslot[0];
    }
}

// Adjoint seeds of  sum_k w_KE,k KE_k + w_R,k runout_k  at the final step
// (small[16 k + 5..6] = weights), and zeroed history and parameter adjoints.
__global__ void __launch_bounds__(TILE) k_adj_seed(Dev d, AdjBufs a, const HostInstLo* __restrict__ hl)
{
    const size_t plane = (size_t)d.Lmax * d.ncap;
    for_live_slots(d, [&](int s, int k, const InstD& D) {
        const double* sm = d.small + 16 * k;
        const float wke = (float)sm[5], wro = (float)sm[6];
        const float4 v = d.outV[s], w = d.outW[s];
        const float m = d.omg[D.cur][s].w;
        const int4 p = d.pos[D.cur][s];
        const float r = (float)(p.w * hl[k].q);
        const float I = 0.4f * m * r * r;
        float4 xb = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((int)sm[4] == s && sm[3] > 0.0) {
            const double x = hl[k].lo[0] + (double)p.x * hl[k].q - sm[0];
            const double y = hl[k].lo[1] + (double)p.y * hl[k].q - sm[1];
            xb.x = (float)(wro * x / sm[3]);
            xb.y = (float)(wro * y / sm[3]);
        }
        a.xb[s] = xb;
        a.vb[s] = make_float4(wke * m * v.x, wke * m * v.y, wke * m * v.z, 0.f);
        a.wb[s] = make_float4(wke * I * w.x, wke * I * w.y, wke * I * w.z, 0.f);
        a.wxib[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int e = 0; e < d.Lmax; ++e)
            for (int c3 = 0; c3 < 3; ++c3) a.xib[c3 * plane + (size_t)e * d.ncap + s] = 0.f;
        a.thb[3 * (size_t)s] = a.thb[3 * (size_t)s + 1] = a.thb[3 * (size_t)s + 2] = 0.0;
    });
}

// per-instance sum of the parameter adjoints (fixed order) into small[16 k + 8..10]
__global__ void __launch_bounds__(256) k_adj_reduce(Dev d, AdjBufs a)
{
    const int k = blockIdx.x;
    const InstC& c = d.ic[k];
    const int n = d.id[k].n;
    __shared__ double sh[3][256];
    double t[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int q3 = 0; q3 < 3; ++q3) t[q3] += a.thb[3 * (size_t)(c.slot0 + i) + q3];
    for (int q3 = 0; q3 < 3; ++q3) sh[q3][threadIdx.x] = t[q3];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q3 = 0; q3 < 3; ++q3) sh[q3][threadIdx.x] += sh[q3][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q3 = 0; q3 < 3; ++q3) d.small[16 * k + 8 + q3] = sh[q3][0];
}

}  // namespace

// ============================================================== host side


namespace cgdem {

thread_local std::string g_cfg_err = "no error";

dem_status fail(dem_ctx* c, dem_status st, const std::string& msg)
{
    if (c) c->err = msg;
    return st;
}


struct Layout {
    size_t total = 0;
    size_t take(size_t bytes)
    {
        size_t o = total;
        total += (bytes + 255) & ~size_t(255);
        return o;
    }
};

struct Plan {
    std::vector<InstC> ic;
    std::vector<HostInstLo> hl;
    std::vector<unsigned> spread;
    std::vector<int> tile_inst;
    std::vector<int> part_inst;
    std::vector<long long> count;
    int ncap = 0, ntiles = 0, Lmax = 0, B = 0;
    unsigned ncodes = 0, nparts = 0;
    // offsets
    size_t o_pos[2], o_vel[2], o_omg[2], o_nbr[2], o_hist[2], o_cnt[2], o_hmask[2], o_fext[2], o_whist[2], o_wseg[2], o_wrem;
    size_t o_cellcode, o_cslot, o_perm, o_fin, o_spos, o_sid, o_ccount, o_crange, o_part, o_pinst, o_soi, o_tile, o_live, o_ic, o_id, o_spread, o_g,
        o_goff, o_outF, o_outT, o_outV, o_outW, o_outWX, o_xi, o_cmask, o_stage, o_hl, o_small, o_wgeo;
    size_t bytes = 0;
};

int ceil_log2(long long v)
{
    int b = 0;
    while ((1ll << b) < v) ++b;
    return b;
}

dem_status make_plan(const dem_config* cfg, Plan& p, std::string& err)
{
    if (!cfg || cfg->n_instances < 1 || !cfg->inst) { err = "config needs n_instances >= 1"; return DEM_ERR_ARG; }
    if (cfg->max_neighbors < 1 || cfg->max_neighbors > MAXL) { err = "max_neighbors must be in 1..32"; return DEM_ERR_ARG; }
    p.B = cfg->n_instances;
    p.Lmax = cfg->max_neighbors;
    long long slot = 0;
    unsigned code = 0;
    for (int k = 0; k < p.B; ++k) {
        const dem_instance_desc& s = cfg->inst[k];
        char buf[256];
        if (s.n < 0 || s.capacity < s.n || s.capacity < 1) { snprintf(buf, sizeof buf, "instance %d: need 0 <= n <= capacity, capacity >= 1", k); err = buf; return DEM_ERR_ARG; }
        if (s.periodic[2]) { snprintf(buf, sizeof buf, "instance %d: z cannot be periodic", k); err = buf; return DEM_ERR_ARG; }
        if (!(s.dt > 0) || !(s.skin > 0) || !(s.r_max > 0) || !(s.E > 0) || !(s.e > 0 && s.e <= 1) || !(s.mu >= 0) ||
            !(s.nu > -1 && s.nu < 0.5) || !(s.rho > 0)) {
            snprintf(buf, sizeof buf, "instance %d: dt, skin, r_max, E, rho > 0; 0 < e <= 1; mu >= 0; -1 < nu < 0.5", k);
            err = buf;
            return DEM_ERR_ARG;
        }
        double ext[3], emax = 0;
        for (int a = 0; a < 3; ++a) {
            ext[a] = s.hi[a] - s.lo[a];
            if (!(ext[a] > 0)) { snprintf(buf, sizeof buf, "instance %d: empty box", k); err = buf; return DEM_ERR_ARG; }
            emax = std::max(emax, ext[a]);
        }
        // quantum: smallest power of two with emax / q <= 2^30
        int e2 = (int)std::ceil(std::log2(emax / 1073741824.0));
        double q = std::ldexp(1.0, e2);
        while (emax / q > 1073741824.0) q *= 2.0;
        InstC c{};
        HostInstLo h{};
        c.slot0 = (int)slot;
        c.cap = (int)s.capacity;
        const long long rmax_u = (long long)std::ceil(s.r_max / q);
        const long long skin_u = (long long)std::llround(s.skin / q);
        const long long hcell = 2 * rmax_u + skin_u;
        for (int a = 0; a < 3; ++a) {
            long long eu = (long long)std::llround(ext[a] / q);
            c.ext[a] = (int)eu;
            c.per[a] = s.periodic[a] ? 1 : 0;
            c.half[a] = (int)(eu / 2);
            long long n = eu / hcell;
            if (c.per[a] && n < 3) { snprintf(buf, sizeof buf, "instance %d: periodic axis %d shorter than 3 cells (2 r_max + skin)", k, a); err = buf; return DEM_ERR_ARG; }
            if (n < 1) n = 1;
            if (n > 4096) n = 4096;
            c.nc[a] = (int)n;
            h.lo[a] = s.lo[a];
        }
        int bits[3], tb = 0;
        for (int a = 0; a < 3; ++a) { bits[a] = ceil_log2(c.nc[a]); tb += bits[a]; }
        if (tb > 28) { snprintf(buf, sizeof buf, "instance %d: cell grid too large", k); err = buf; return DEM_ERR_ARG; }
        // Morton spread tables
        int pos_of[3][32];
        {
            int pos = 0;
            for (int b = 0; b < 32; ++b)
                for (int a = 0; a < 3; ++a)
                    if (b < bits[a]) pos_of[a][b] = pos++;
        }
        for (int a = 0; a < 3; ++a) {
            c.spread_off[a] = (int)p.spread.size();
            for (int v = 0; v < c.nc[a]; ++v) {
                unsigned sv = 0;
                for (int b = 0; b < bits[a]; ++b)
                    if ((v >> b) & 1) sv |= 1u << pos_of[a][b];
                p.spread.push_back(sv);
            }
        }
        code = (code + SCAN_TILE - 1) / SCAN_TILE * SCAN_TILE;   // scan chunks never straddle instances
        c.code0 = (int)code;
        c.ncode = 1 << tb;
        code += (unsigned)c.ncode;
        c.floor_on = s.floor_on ? 1 : 0;
        c.zrem = INT_MIN;   // no removal height until dem_set_walls gives one
        c.skin = (int)skin_u;
        c.skin_f = (float)skin_u;
        c.clamp_fn = s.clamp_fn ? 1 : 0;
        c.q = (float)q;
        c.dt = (float)s.dt;
        c.dt_over_q = (float)(s.dt / q);
        for (int a = 0; a < 3; ++a) { c.g[a] = (float)s.g[a]; c.floor_v[a] = (float)s.floor_v[a]; }
        const double nu = s.nu, E = s.E;
        const double Eeff = 1.0 / (2.0 * (1.0 - nu * nu) / E);
        const double Geff = 1.0 / (2.0 * 2.0 * (2.0 - nu) * (1.0 + nu) / E);
        const double le = std::log(s.e);
        const double beta = le / std::sqrt(le * le + M_PI * M_PI);
        c.c_kn = (float)(4.0 / 3.0 * Eeff);
        c.c_kt = (float)(8.0 * Geff);
        c.nbeta = (float)(-beta);
        c.mu = (float)s.mu;
        c.mu_w = (float)(s.mu_wall < 0 ? s.mu : s.mu_wall);
        c.gt_ratio = (float)std::sqrt(2.0 * (8.0 * Geff) / (3.0 * (4.0 / 3.0 * Eeff)));
        c.mu_w_follows = s.mu_wall < 0 ? 1 : 0;
        c.inv_E = (float)(1.0 / E);
        // beta = ln e / sqrt(ln^2 e + pi^2): dbeta/de = pi^2 / (e (ln^2 e + pi^2)^(3/2))
        c.dnb_de = (float)(-(M_PI * M_PI) / (s.e * std::pow(le * le + M_PI * M_PI, 1.5)));
        h.q = q;
        h.rho = s.rho;
        p.ic.push_back(c);
        p.hl.push_back(h);
        p.count.push_back(s.n);
        // whole pairs of tiles: a step block of 2 TILE threads never straddles two instances
        const long long tiles = 2 * ((s.capacity + 2 * TILE - 1) / (2 * TILE));
        for (long long t = 0; t < tiles; ++t) p.tile_inst.push_back(k);
        slot += tiles * TILE;
        if (slot > (1ll << 30)) { err = "total capacity too large"; return DEM_ERR_ARG; }
    }
    p.ncap = (int)slot;
    p.ntiles = (int)(slot / TILE);
    p.ncodes = code;
    p.nparts = (code + SCAN_TILE - 1) / SCAN_TILE;
    p.part_inst.assign(std::max(1u, p.nparts), -1);
    for (int k = 0; k < p.B; ++k)
        for (unsigned b = (unsigned)p.ic[k].code0 / SCAN_TILE;
             b < ((unsigned)p.ic[k].code0 + (unsigned)p.ic[k].ncode + SCAN_TILE - 1) / SCAN_TILE; ++b)
            p.part_inst[b] = k;
    Layout L;
    const size_t N = (size_t)p.ncap, Lm = (size_t)p.Lmax;
    for (int b = 0; b < 2; ++b) {
        p.o_pos[b] = L.take(N * 16);
        p.o_vel[b] = L.take(N * 16);
        p.o_omg[b] = L.take(N * 16);
        p.o_nbr[b] = L.take(N * Lm * 4);
        p.o_hist[b] = L.take(N * Lm * 12);
        p.o_cnt[b] = L.take(N * 4);
        p.o_hmask[b] = L.take(N * 4);
        p.o_fext[b] = L.take(N * 16);
        p.o_whist[b] = L.take(N * 16);
        p.o_wseg[b] = L.take(N * 32);
    }
    p.o_wrem = L.take(sizeof(double) * 2 * p.B);
    p.o_cellcode = L.take(N * 4);
    p.o_cslot = L.take(N * 4);
    p.o_perm = L.take(N * 4);
    p.o_fin = L.take(N * 4);
    p.o_spos = L.take(N * 16);
    p.o_sid = L.take(N * 4);
    p.o_ccount = L.take((size_t)p.ncodes * 4);
    p.o_crange = L.take((size_t)p.ncodes * 8);
    p.o_part = L.take((size_t)std::max(1u, p.nparts) * 4);
    p.o_pinst = L.take((size_t)std::max(1u, p.nparts) * 4);
    p.o_soi = L.take(N * 4);
    p.o_tile = L.take((size_t)p.ntiles * 4);
    p.o_live = L.take((size_t)p.ntiles * 4);
    p.o_ic = L.take(sizeof(InstC) * p.B);
    p.o_id = L.take(sizeof(InstD) * p.B);
    p.o_spread = L.take(p.spread.size() * 4);
    p.o_g = L.take(sizeof(Glob));
    p.o_goff = L.take(sizeof(long long) * (p.B + 1));
    p.o_outF = L.take(N * 16);
    p.o_outT = L.take(N * 16);
    p.o_outV = L.take(N * 16);
    p.o_outW = L.take(N * 16);
    p.o_outWX = L.take(N * 16);
    p.o_xi = L.take(N * Lm * 12);
    p.o_cmask = L.take(N * 8);
    p.o_stage = L.take(N * 24);
    p.o_hl = L.take(sizeof(HostInstLo) * p.B);
    p.o_small = L.take(sizeof(double) * 16 * p.B);
    p.o_wgeo = L.take(sizeof(WallGeo) * p.B);
    p.bytes = L.total;
    return DEM_OK;
}

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

dem_status upload_goff(dem_ctx* ctx)
{
    std::vector<long long> goff(ctx->B + 1, 0);
    for (int k = 0; k < ctx->B; ++k) goff[k + 1] = goff[k] + ctx->count[k];
    CU(cudaMemcpyAsync(ctx->dev.goff, goff.data(), sizeof(long long) * (ctx->B + 1), cudaMemcpyHostToDevice,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

// the host copy of the IDs handed out per instance, after coupling calls changed them on the
// device (synchronises; also takes in the device status)
dem_status refresh_count(dem_ctx* ctx)
{
    if (!ctx->count_stale) return DEM_OK;
    std::vector<InstD> D(ctx->B);
    CU(cudaMemcpyAsync(D.data(), ctx->dev.id, sizeof(InstD) * ctx->B, cudaMemcpyDeviceToHost, ctx->stream));
    unsigned stv = 0;
    CU(cudaMemcpyAsync(&stv, &ctx->dev.g->status, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < ctx->B; ++k) ctx->count[k] = D[k].nid;
    ctx->count_stale = false;
    ctx->status |= stv;
    return check_status(ctx);
}

long long total_count(const dem_ctx* ctx)
{
    long long t = 0;
    for (long long c : ctx->count) t += c;
    return t;
}

dem_status check_status(dem_ctx* ctx)
{
    if (!ctx->status) return DEM_OK;
    if (ctx->status & ST_NONFINITE) return fail(ctx, DEM_ERR_NONFINITE, "non-finite force, torque or velocity on the device");
    if (ctx->status & ST_ESCAPED) return fail(ctx, DEM_ERR_ESCAPED, "a particle left the representable range");
    if (ctx->status & ST_CAPACITY) return fail(ctx, DEM_ERR_CAPACITY, "neighbour list wider than max_neighbors");
    if (ctx->status & ST_TIMEOUT) return fail(ctx, DEM_ERR_TIMEOUT, "a bounded device wait gave up");
    if (ctx->status & ST_TRUNC) return fail(ctx, DEM_ERR_CAPACITY, "more contacts than the output width");
    if (ctx->status & ST_INSERT) return fail(ctx, DEM_ERR_CAPACITY, "inserted particles exceed the fine level's capacity");
    if (ctx->status & ST_BOUNDS) {
        // where the check fired (read synchronously: an error path)
        Glob gl{};
        cudaStreamSynchronize(ctx->stream);
        cudaMemcpy(&gl, ctx->dev.g, sizeof(Glob), cudaMemcpyDeviceToHost);
        return fail(ctx, DEM_ERR_BOUNDS,
                    "an index out of range (bounds-checked build): check " + std::to_string(gl.err_site) + ", slot " +
                        std::to_string(gl.err_slot) + ", index " + std::to_string(gl.err_val) + " (capacity " +
                        std::to_string(ctx->ncap) + ")");
    }
    if (ctx->status & ST_SKIN)
        return fail(ctx, DEM_ERR_CAPACITY,
                    "a particle moved more than half the skin while the lists were frozen for a differentiable "
                    "rollout: use a larger skin");
    return DEM_ERR_STATE;
}

int step_block(const dem_ctx* ctx);

// launch the rebuild chain (each kernel returns at once when no instance is flagged)
dem_status launch_rebuild(dem_ctx* ctx, cudaStream_t st)
{
    const Dev& d = ctx->dev;
    const unsigned gt = (unsigned)ctx->grid_rb;
    k_rb_clear<<<std::min(std::max(1u, ctx->nparts), 152u * 8u), 256, 0, st>>>(d);
    k_rb_bin<<<gt, TILE, 0, st>>>(d);
    k_scan_reduce<<<std::max(1u, ctx->nparts), SCAN_T, 0, st>>>(d);
    k_scan_top<<<1, 1024, 0, st>>>(d);
    k_scan_down<<<std::max(1u, ctx->nparts), SCAN_T, 0, st>>>(d);
    k_rb_scatter<<<gt, TILE, 0, st>>>(d);
    k_rb_cellsort<<<gt, TILE, 0, st>>>(d);
    k_rb_count<<<1, 256, 0, st>>>(d);
    if (step_block(ctx) == SMW_BS)
        k_rb_winsort<SMW_SORT_W><<<gt, WS_T, 0, st>>>(d, ctx->grid_smw);
    else
        k_rb_tilesort<<<gt, TILE, 0, st>>>(d);
    if (ctx->list_staged)
        k_rb_build<true><<<ctx->grid_build_staged, RB_T, 0, st>>>(d);
    else
        k_rb_build<false><<<ctx->grid_build, RB_T, 0, st>>>(d);
    k_rb_finish<<<1, 256, 0, st>>>(d);          // 256 threads: its shared arrays
    CU(cudaGetLastError());
    return DEM_OK;
}

dem_status launch_eval(dem_ctx* ctx)
{
    dem_status st = launch_rebuild(ctx, ctx->stream);
    if (st) return st;
    k_step<1, true><<<ctx->grid1, TILE, 0, ctx->stream>>>(ctx->dev, ctx->fresh ? 1 : 0, 0, 0);
    CU(cudaGetLastError());
    return DEM_OK;
}

// mark every instance for a rebuild with cleared histories (fresh state)
__global__ void k_mark_fresh(Dev d)
{
    for (int k = threadIdx.x; k < d.B; k += blockDim.x) {
        d.id[k].flag = 2;
        d.id[k].disp = 0.f;
        d.id[k].stepmax = 0u;
    }
    if (threadIdx.x == 0) d.g->any = 1u;
}

void destroy_graph(dem_ctx* ctx)
{
    for (cudaEvent_t e : ctx->ev0) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->ev1) cudaEventDestroy(e);
    ctx->ev0.clear();
    ctx->ev1.clear();
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    if (ctx->rb_graph) cudaGraphDestroy(ctx->rb_graph);
    ctx->gexec = nullptr;
    ctx->graph = nullptr;
    ctx->rb_graph = nullptr;
}

// the step kernel's block size: the one set, else SM-wide blocks for a single instance with
// one lane per particle whose live rows give every resident warp at least SMW_MIN slices (below
// that the last slices' quantisation dominates, and 128-thread blocks are as fast), else 128
constexpr int SMW_MIN = 4;
int step_block(const dem_ctx* ctx)
{
    if (ctx->step_bs) return ctx->step_bs;
    if (ctx->step_lanes == 1 && ctx->B == 1 && ctx->grid_smw > 0 &&
        ctx->count[0] >= (long long)SMW_MIN * ctx->grid_smw * (SMW_BS / 32) * 32)
        return SMW_BS;
    return TILE;
}

// dynamic shared memory of the step kernel (the SM-wide block's staging slots)
unsigned step_smem(const dem_ctx* ctx) { return step_block(ctx) == SMW_BS ? 2 * 2 * SMW_BS * sizeof(float4) : 0u; }

// the step kernel (MODE 0) at the context's block size, and its persistent grid
void* step_func(const dem_ctx* ctx)
{
    switch (ctx->step_lanes) {
    case 2: return ctx->walls ? (void*)k_step<0, true, 128, 2> : (void*)k_step<0, false, 128, 2>;
    case 4: return ctx->walls ? (void*)k_step<0, true, 128, 4> : (void*)k_step<0, false, 128, 4>;
    case 8: return ctx->walls ? (void*)k_step<0, true, 128, 8> : (void*)k_step<0, false, 128, 8>;
    default: break;
    }
    switch (step_block(ctx)) {
    case SMW_BS: return ctx->walls ? (void*)k_step<0, true, SMW_BS> : (void*)k_step<0, false, SMW_BS>;
    case 64: return ctx->walls ? (void*)k_step<0, true, 64> : (void*)k_step<0, false, 64>;
    case 256: return ctx->walls ? (void*)k_step<0, true, 256> : (void*)k_step<0, false, 256>;
    default: return ctx->walls ? (void*)k_step<0, true, 128> : (void*)k_step<0, false, 128>;
    }
}

int step_grid(const dem_ctx* ctx)
{
    if (ctx->step_lanes > 1) return ctx->grid_lanes[ctx->step_lanes == 2 ? 0 : ctx->step_lanes == 4 ? 1 : 2];
    const int bs = step_block(ctx);
    if (bs == SMW_BS) return ctx->grid_smw;
    return ctx->grid_bs[bs == 64 ? 0 : bs == 256 ? 2 : 1];
}

dem_status launch_step(dem_ctx* ctx, int prime)
{
    Dev dv = ctx->dev;
    cudaGraphConditionalHandle h = 0;
    int use_cond = 0;
    void* args[] = {&dv, &prime, &h, &use_cond};
    CU(cudaLaunchKernel(step_func(ctx), dim3(step_grid(ctx)), dim3(step_block(ctx)), args, step_smem(ctx), ctx->stream));
    return DEM_OK;
}

constexpr int EV_EVERY = 5;    // step kernels per timed one in a graph

// the fused step kernel for the context's walls and lanes per particle
void* fused_func(const dem_ctx* ctx)
{
    switch (ctx->step_lanes) {
    case 2: return ctx->walls ? (void*)k_steps<true, 2> : (void*)k_steps<false, 2>;
    case 4: return ctx->walls ? (void*)k_steps<true, 4> : (void*)k_steps<false, 4>;
    case 8: return ctx->walls ? (void*)k_steps<true, 8> : (void*)k_steps<false, 8>;
    default: return ctx->walls ? (void*)k_steps<true, 1> : (void*)k_steps<false, 1>;
    }
}

// A graph of S steps run by fused launches: init (S steps to do, pending list build) ->
// while (steps remain) { if (list build needed) rebuild chain; k_steps }, with CUDA events
// around the loop.
dem_status build_fused_graph(dem_ctx* ctx, cudaGraph_t g, int S)
{
    cudaGraphConditionalHandle h_loop, h_rb;
    CU(cudaGraphConditionalHandleCreate(&h_loop, g, 0, 0));
    CU(cudaGraphConditionalHandleCreate(&h_rb, g, 0, 0));
    Dev dv = ctx->dev;
    long long SS = S;
    cudaGraphNode_t init;
    {
        void* args[] = {&dv, &SS, &h_rb, &h_loop};
        cudaKernelNodeParams kp{};
        kp.func = (void*)k_steps_init;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1);
        kp.kernelParams = args;
        CU(cudaGraphAddKernelNode(&init, g, nullptr, 0, &kp));
    }
    ctx->ev0.resize(1);
    ctx->ev1.resize(1);
    CU(cudaEventCreate(&ctx->ev0[0]));
    CU(cudaEventCreate(&ctx->ev1[0]));
    cudaGraphNode_t e0, e1, loop;
    CU(cudaGraphAddEventRecordNode(&e0, g, &init, 1, ctx->ev0[0]));
    cudaGraphNodeParams wp{};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    CU(cudaGraphAddNode(&loop, g, &e0, nullptr, 1, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    cudaGraphNodeParams ip{};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = h_rb;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t ifn, child, kn;
    CU(cudaGraphAddNode(&ifn, body, nullptr, nullptr, 0, &ip));
    CU(cudaGraphAddChildGraphNode(&child, ip.conditional.phGraph_out[0], nullptr, 0, ctx->rb_graph));
    {
        void* args[] = {&dv, &h_rb, &h_loop};
        cudaKernelNodeParams kp{};
        kp.func = fused_func(ctx);
        kp.gridDim = dim3(std::min(ctx->ntiles * ctx->step_lanes, ctx->grid_fused));   // all resident: cooperative
        kp.blockDim = dim3(TILE);
        kp.kernelParams = args;
        CU(cudaGraphAddKernelNode(&kn, body, &ifn, 1, &kp));
        cudaLaunchAttributeValue coop{};
        coop.cooperative = 1;
        CU(cudaGraphKernelNodeSetAttribute(kn, cudaLaunchAttributeCooperative, &coop));
    }
    CU(cudaGraphAddEventRecordNode(&e1, g, &loop, 1, ctx->ev1[0]));
    CU(cudaGraphInstantiate(&ctx->gexec, g, 0));
    ctx->graph_steps = S;
    ctx->graph_fused = true;
    return DEM_OK;
}

dem_status build_graph(dem_ctx* ctx, int S)
{
    destroy_graph(ctx);
    if (S <= 0) return DEM_OK;
    // the rebuild chain, captured once
    cudaStream_t cs;
    CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    dem_status st = launch_rebuild(ctx, cs);
    cudaGraph_t rb = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &rb);
    cudaStreamDestroy(cs);
    if (st) return st;
    if (ce != cudaSuccess) return fail(ctx, DEM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
    ctx->rb_graph = rb;
    cudaGraph_t g;
    CU(cudaGraphCreate(&g, 0));
    ctx->graph = g;
    ctx->graph_fused = false;
    {
        // fused steps: one cooperative launch runs the steps between list builds; chosen by
        // default when a block for every tile holding live slots fits on the GPU at once
        int nsm = 0, occ = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fused_func(ctx), TILE, 0);
        cudaGetLastError();
        ctx->grid_fused = nsm * occ;
        const bool can = (ctx->step_bs == 0 || ctx->step_bs == TILE) && ctx->grid_fused > 0;
        if (ctx->graph_mode == 2 && !can) return fail(ctx, DEM_ERR_STATE, "fused steps need 128-thread blocks");
        // the tiles holding live slots (from the host's last copy of the counts)
        long long live = 0;
        for (int k = 0; k < ctx->B; ++k) live += 2 * ((ctx->count[k] + 2 * TILE - 1) / (2 * TILE));
        if (ctx->graph_mode == 2 || (ctx->graph_mode == 0 && can && live * ctx->step_lanes <= ctx->grid_fused))
            return build_fused_graph(ctx, g, S);
    }
    std::vector<cudaGraphConditionalHandle> h(S);
    for (int i = 0; i < S; ++i) CU(cudaGraphConditionalHandleCreate(&h[i], g, 0, 0));
    Dev dv = ctx->dev;
    cudaGraphNode_t prev;
    {
        cudaKernelNodeParams kp{};
        void* args[] = {&dv, &h[0]};
        kp.func = (void*)k_set_cond;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1);
        kp.kernelParams = args;
        CU(cudaGraphAddKernelNode(&prev, g, nullptr, 0, &kp));
    }
    // CUDA events around every EV_EVERY-th step kernel (each pair of event nodes adds a few
    // microseconds to the step, so the timing is sampled)
    const int nev = (S + EV_EVERY - 1) / EV_EVERY;
    ctx->ev0.resize(nev);
    ctx->ev1.resize(nev);
    for (int i = 0; i < nev; ++i) {
        CU(cudaEventCreate(&ctx->ev0[i]));
        CU(cudaEventCreate(&ctx->ev1[i]));
    }
    for (int i = 0; i < S; ++i) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h[i];
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t cn;
        CU(cudaGraphAddNode(&cn, g, &prev, nullptr, 1, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t child;
        CU(cudaGraphAddChildGraphNode(&child, body, nullptr, 0, rb));
        int prime = 0;
        int use_cond = i + 1 < S ? 1 : 0;
        cudaGraphConditionalHandle hn = i + 1 < S ? h[i + 1] : h[i];
        void* args[] = {&dv, &prime, &hn, &use_cond};
        cudaKernelNodeParams kp{};
        kp.func = step_func(ctx);
        kp.gridDim = dim3(step_grid(ctx));
        kp.blockDim = dim3(step_block(ctx));
        kp.sharedMemBytes = step_smem(ctx);
        kp.kernelParams = args;
        cudaGraphNode_t kn;
        if (i % EV_EVERY == 0) {
            cudaGraphNode_t e0, e1;
            CU(cudaGraphAddEventRecordNode(&e0, g, &cn, 1, ctx->ev0[i / EV_EVERY]));
            CU(cudaGraphAddKernelNode(&kn, g, &e0, 1, &kp));
            CU(cudaGraphAddEventRecordNode(&e1, g, &kn, 1, ctx->ev1[i / EV_EVERY]));
            prev = e1;
        } else {
            CU(cudaGraphAddKernelNode(&kn, g, &cn, 1, &kp));
            prev = kn;
        }
    }
    CU(cudaGraphInstantiate(&ctx->gexec, g, 0));
    ctx->graph_steps = S;
    return DEM_OK;
}

}  // namespace cgdem

namespace cgdem {
// error text reported by dem_last_error(NULL) for calls made without a context
void set_thread_error(const std::string& msg) { g_cfg_err = msg; }
}  // namespace cgdem

// ============================================================== grid fields
// Volume averages of one instance on a uniform grid: per cell the solid volume of the
// particles whose centres lie in it, their mass and momentum (velocities at the current
// step, as reconstructed by the read-out evaluation); particles marked for removal are left out.
namespace {
__global__ void __launch_bounds__(256) k_grid_sums(Dev d, int k, const HostInstLo* __restrict__ hl, double lx, double ly,
                                                   double lz, double h, int n0, int n1, int n2, double* __restrict__ out)
{
    const InstC& c = d.ic[k];
    const InstD D = d.id[k];
    const double q = hl[k].q;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D.n; i += gridDim.x * blockDim.x) {
        const int s = c.slot0 + i;
        if (__float_as_uint(d.vel[D.cur][s].w) & GONE_BIT) continue;
        const int4 P = d.pos[D.cur][s];
        const long long ix = (long long)floor((hl[k].lo[0] + (double)P.x * q - lx) / h);
        const long long iy = (long long)floor((hl[k].lo[1] + (double)P.y * q - ly) / h);
        const long long iz = (long long)floor((hl[k].lo[2] + (double)P.z * q - lz) / h);
        if (ix < 0 || iy < 0 || iz < 0 || ix >= n0 || iy >= n1 || iz >= n2) continue;
        double* o = out + 5 * ((iz * n1 + iy) * (long long)n0 + ix);
        const double m = d.omg[D.cur][s].w, r = (double)P.w * q;
        const float4 v = d.outV[s];
        atomicAdd(o, 4.0 / 3.0 * 3.14159265358979323846 * r * r * r);
        atomicAdd(o + 1, m);
        atomicAdd(o + 2, m * v.x);
        atomicAdd(o + 3, m * v.y);
        atomicAdd(o + 4, m * v.z);
    }
}

__global__ void k_grid_finish(double* __restrict__ out, long long ncell, double cellvol)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell; i += (long long)gridDim.x * blockDim.x) {
        double* o = out + 5 * i;
        const double m = o[1];
        o[0] /= cellvol;
        for (int a = 0; a < 3; ++a) o[2 + a] = m > 0.0 ? o[2 + a] / m : 0.0;
    }
}
}  // namespace

// ================================================================== C ABI

extern "C" {

dem_status dem_query_workspace(const dem_config* cfg, int64_t* bytes_out)
{
    if (!bytes_out) return DEM_ERR_ARG;
    Plan p;
    dem_status st = make_plan(cfg, p, g_cfg_err);
    if (st) return st;
    *bytes_out = (int64_t)p.bytes;
    return DEM_OK;
}

dem_status dem_create(const dem_config* cfg, void* workspace, int64_t workspace_bytes, void* stream, dem_ctx** out)
{
    if (!out) return DEM_ERR_ARG;
    *out = nullptr;
    Plan p;
    dem_status st = make_plan(cfg, p, g_cfg_err);
    if (st) return st;
    if (!workspace || (size_t)workspace_bytes < p.bytes || ((uintptr_t)workspace & 255)) {
        g_cfg_err = "workspace missing, too small or not 256-byte aligned";
        return DEM_ERR_ARG;
    }
    dem_ctx* ctx = new dem_ctx();
    ctx->stream = (cudaStream_t)stream;
    cudaGetDevice(&ctx->device);
    ctx->B = p.B;
    ctx->Lmax = p.Lmax;
    ctx->ncap = p.ncap;
    ctx->ntiles = p.ntiles;
    ctx->ncodes = p.ncodes;
    ctx->nparts = p.nparts;
    ctx->ic = p.ic;
    ctx->hl = p.hl;
    for (int k = 0; k < p.B; ++k) {
        ctx->nu.push_back(cfg->inst[k].nu);
        ctx->rmax.push_back(cfg->inst[k].r_max);
    }
    ctx->count = p.count;
    char* base = (char*)workspace;
    Dev& d = ctx->dev;
    for (int b = 0; b < 2; ++b) {
        d.pos[b] = (int4*)(base + p.o_pos[b]);
        d.vel[b] = (float4*)(base + p.o_vel[b]);
        d.omg[b] = (float4*)(base + p.o_omg[b]);
        d.nbr[b] = (int*)(base + p.o_nbr[b]);
        d.hist[b] = (float*)(base + p.o_hist[b]);
        d.cnt[b] = (int*)(base + p.o_cnt[b]);
        d.hmask[b] = (unsigned*)(base + p.o_hmask[b]);
        d.fext[b] = (float4*)(base + p.o_fext[b]);
        d.whist[b] = (float4*)(base + p.o_whist[b]);
        d.wseg[b] = (float4*)(base + p.o_wseg[b]);
    }
    d.wrem = (double*)(base + p.o_wrem);
    d.cellcode = (unsigned*)(base + p.o_cellcode);
    d.cslot = (unsigned*)(base + p.o_cslot);
    d.perm = (int*)(base + p.o_perm);
    d.fin = (int*)(base + p.o_fin);
    d.spos = (int4*)(base + p.o_spos);
    d.sid = (int*)(base + p.o_sid);
    d.ccount = (unsigned*)(base + p.o_ccount);
    d.crange = (uint2*)(base + p.o_crange);
    d.part = (unsigned*)(base + p.o_part);
    d.part_inst = (int*)(base + p.o_pinst);
    d.slot_of_id = (int*)(base + p.o_soi);
    d.tile_inst = (int*)(base + p.o_tile);
    d.live_tiles = (int*)(base + p.o_live);
    d.ic = (const InstC*)(base + p.o_ic);
    d.id = (InstD*)(base + p.o_id);
    d.spread = (const unsigned*)(base + p.o_spread);
    d.g = (Glob*)(base + p.o_g);
    d.goff = (long long*)(base + p.o_goff);
    d.outF = (float4*)(base + p.o_outF);
    d.outT = (float4*)(base + p.o_outT);
    d.outV = (float4*)(base + p.o_outV);
    d.outW = (float4*)(base + p.o_outW);
    d.outWX = (float4*)(base + p.o_outWX);
    d.xi_out = (float*)(base + p.o_xi);
    d.cmask = (unsigned long long*)(base + p.o_cmask);
    d.stage = (double*)(base + p.o_stage);
    ctx->d_hl = (HostInstLo*)(base + p.o_hl);
    d.small = (double*)(base + p.o_small);
    d.wgeo = (const WallGeo*)(base + p.o_wgeo);
    d.ncap = p.ncap;
    d.ntiles = p.ntiles;
    d.B = p.B;
    d.Lmax = p.Lmax;
    d.ncodes = p.ncodes;
    d.nparts = p.nparts;
    std::vector<InstD> idv(p.B);
    for (int k = 0; k < p.B; ++k) {
        idv[k] = InstD{};
        idv[k].n = (int)p.count[k];
        idv[k].nid = (int)p.count[k];
        idv[k].flag = 2;
    }
    Glob gl{};
    gl.any = 1u;
    gl.nlive = p.ntiles;
    cudaStream_t s = ctx->stream;
#define CUC(call)                                                    \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) {                                     \
            delete ctx;                                              \
            return DEM_ERR_CUDA;                                     \
        }                                                            \
    } while (0)
    CUC(cudaMemcpyAsync((void*)d.ic, p.ic.data(), sizeof(InstC) * p.B, cudaMemcpyHostToDevice, s));
    CUC(cudaMemcpyAsync(d.id, idv.data(), sizeof(InstD) * p.B, cudaMemcpyHostToDevice, s));
    CUC(cudaMemcpyAsync((void*)d.spread, p.spread.data(), p.spread.size() * 4, cudaMemcpyHostToDevice, s));
    CUC(cudaMemcpyAsync(d.tile_inst, p.tile_inst.data(), p.tile_inst.size() * 4, cudaMemcpyHostToDevice, s));
    std::vector<int> all_tiles(p.ntiles);              // until the first list build: every tile
    for (int t = 0; t < p.ntiles; ++t) all_tiles[t] = t;
    CUC(cudaMemcpyAsync(d.live_tiles, all_tiles.data(), all_tiles.size() * 4, cudaMemcpyHostToDevice, s));
    CUC(cudaMemcpyAsync(d.part_inst, p.part_inst.data(), p.part_inst.size() * 4, cudaMemcpyHostToDevice, s));
    CUC(cudaMemcpyAsync(d.g, &gl, sizeof(Glob), cudaMemcpyHostToDevice, s));
    CUC(cudaMemcpyAsync(ctx->d_hl, p.hl.data(), sizeof(HostInstLo) * p.B, cudaMemcpyHostToDevice, s));
    CUC(cudaMemsetAsync(d.hist[0], 0, (size_t)p.ncap * p.Lmax * 12, s));
    CUC(cudaMemsetAsync(d.hist[1], 0, (size_t)p.ncap * p.Lmax * 12, s));
    CUC(cudaMemsetAsync(d.wrem, 0, sizeof(double) * 2 * p.B, s));
    k_init_ids<<<nblk(p.ncap, 256), 256, 0, s>>>(d);
    CUC(cudaGetLastError());
    CUC(cudaStreamSynchronize(s));
#undef CUC
    if (upload_goff(ctx)) {
        delete ctx;
        return DEM_ERR_CUDA;
    }
    {
        int nsm = 0, b0 = 0, b1 = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, k_step<0, false>, TILE, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_step<1, true>, TILE, 0);
        ctx->grid0 = std::max(1, std::min(ctx->ntiles, std::max(1, nsm) * std::max(1, b0)));
        {
            // persistent step grids per block size: a wave of blocks, at most one per unit of work
            int bx[3] = {0, 0, 0};
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bx[0], k_step<0, false, 64>, 64, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bx[1], k_step<0, false, 128>, 128, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bx[2], k_step<0, false, 256>, 256, 0);
            const int units[3] = {ctx->ntiles * 2, ctx->ntiles, ctx->ntiles / 2};
            for (int i = 0; i < 3; ++i)
                ctx->grid_bs[i] = std::max(1, std::min(units[i], std::max(1, nsm) * std::max(1, bx[i])));
            // SM-wide blocks (single instance): a block per SM, at most one per tile; 0 if the
            // block does not fit
            if (p.B == 1) {
                const int smem = 2 * 2 * SMW_BS * (int)sizeof(float4);
                int bw = 0;
                if (cudaFuncSetAttribute(k_step<0, false, SMW_BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
                        cudaSuccess &&
                    cudaFuncSetAttribute(k_step<0, true, SMW_BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
                        cudaSuccess)
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bw, k_step<0, false, SMW_BS>, SMW_BS, smem);
                ctx->grid_smw = bw > 0 ? std::min(ctx->ntiles, std::max(1, nsm) * bw) : 0;
            }
            // several lanes per particle (128 threads): LPP times the units of one lane
            int bl[3] = {0, 0, 0};
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl[0], k_step<0, false, 128, 2>, 128, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl[1], k_step<0, false, 128, 4>, 128, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl[2], k_step<0, false, 128, 8>, 128, 0);
            for (int i = 0; i < 3; ++i)
                ctx->grid_lanes[i] = std::max(1, std::min(ctx->ntiles << (i + 1), std::max(1, nsm) * std::max(1, bl[i])));
        }
        ctx->grid1 = std::max(1, std::min(ctx->ntiles, std::max(1, nsm) * std::max(1, b1)));
        ctx->grid_rb = std::max(1, std::min(ctx->ntiles, std::max(1, nsm) * 8));
        int bb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, k_rb_build<false>, RB_T, 0);
        ctx->grid_build = std::max(1, std::min(ctx->ntiles * (TILE / RB_T), std::max(1, nsm) * std::max(1, bb)));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, k_rb_build<true>, RB_T, 0);
        ctx->grid_build_staged = std::max(1, std::min(ctx->ntiles * (TILE / RB_T), std::max(1, nsm) * std::max(1, bb)));
        cudaGetLastError();
    }
    *out = ctx;
    return DEM_OK;
}

dem_status dem_destroy(dem_ctx* ctx)
{
    if (!ctx) return DEM_ERR_ARG;
    cudaStreamSynchronize(ctx->stream);
    destroy_graph(ctx);
    delete ctx;
    return DEM_OK;
}

static bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int field_width(int f)
{
    switch (f) {
    case DEM_F_POS: case DEM_F_VEL: case DEM_F_OMEGA: case DEM_F_FORCE: case DEM_F_TORQUE: case DEM_F_WALL_XI:
    case DEM_F_FEXT: return 3;
    case DEM_F_RADIUS: case DEM_F_MASS: case DEM_F_NBR_COUNT: return 1;
    default: return 0;
    }
}

dem_status dem_write(dem_ctx* ctx, int32_t field, const void* src, int64_t n)
{
    NvtxRange nvtx_range("dem_write");
    if (!ctx) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    const int w = field_width(field);
    if (w == 0 || field == DEM_F_FORCE || field == DEM_F_TORQUE || field == DEM_F_NBR_COUNT)
        return fail(ctx, DEM_ERR_ARG, "field is not writable");
    if (dem_status st = refresh_count(ctx)) return st;
    if (n != total_count(ctx)) return fail(ctx, DEM_ERR_ARG, "n must equal the total particle count");
    if (n == 0) return DEM_OK;
    if (!src) return fail(ctx, DEM_ERR_ARG, "null source");
    const double* dsrc = (const double*)src;
    if (!is_device_ptr(src)) {
        CU(cudaMemcpyAsync(ctx->dev.stage, src, (size_t)n * w * 8, cudaMemcpyHostToDevice, ctx->stream));
        dsrc = ctx->dev.stage;
    }
    if (field == DEM_F_WALL_XI) {            // the floor histories of the lists of this state: build them first
        dem_status st = launch_rebuild(ctx, ctx->stream);
        if (st) return st;
    }
    k_write_field<<<nblk(n, 256), 256, 0, ctx->stream>>>(ctx->dev, field, dsrc, n, ctx->d_hl);
    CU(cudaGetLastError());
    // the held force and the floor histories change neither the lists nor the state's integrity
    if (field != DEM_F_FEXT && field != DEM_F_WALL_XI) {
        k_mark_fresh<<<1, 256, 0, ctx->stream>>>(ctx->dev);
        CU(cudaGetLastError());
        ctx->fresh = true;
        ctx->have_state = true;
    }
    if (dsrc == ctx->dev.stage) CU(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

dem_status dem_read(dem_ctx* ctx, int32_t field, void* dst, int64_t n)
{
    NvtxRange nvtx_range("dem_read");
    if (!ctx) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    const int w = field_width(field);
    if (w == 0) return fail(ctx, DEM_ERR_ARG, "unknown field");
    if (dem_status st = refresh_count(ctx)) return st;
    if (n != total_count(ctx)) return fail(ctx, DEM_ERR_ARG, "n must equal the total particle count");
    if (n == 0) return DEM_OK;
    if (!dst) return fail(ctx, DEM_ERR_ARG, "null destination");
    if (field == DEM_F_VEL || field == DEM_F_OMEGA || field == DEM_F_FORCE || field == DEM_F_TORQUE ||
        field == DEM_F_WALL_XI || field == DEM_F_NBR_COUNT) {
        dem_status st = launch_eval(ctx);
        if (st) return st;
    }
    const bool dev = is_device_ptr(dst);
    double* ddst = dev ? (double*)dst : ctx->dev.stage;
    k_read_field<<<nblk(n, 256), 256, 0, ctx->stream>>>(ctx->dev, field, ddst, n, ctx->d_hl);
    CU(cudaGetLastError());
    if (!dev) {
        CU(cudaMemcpyAsync(dst, ddst, (size_t)n * w * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    return DEM_OK;
}

dem_status dem_read_contacts(dem_ctx* ctx, int32_t* partner, double* xi, int32_t width, int64_t n)
{
    if (!ctx) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    if (ctx->B != 1) return fail(ctx, DEM_ERR_ARG, "contacts I/O needs a single-instance context");
    if (dem_status st = refresh_count(ctx)) return st;
    if (n != total_count(ctx) || width < 1 || !partner || !xi) return fail(ctx, DEM_ERR_ARG, "bad contacts arguments");
    if (!is_device_ptr(partner) || !is_device_ptr(xi)) return fail(ctx, DEM_ERR_ARG, "contacts buffers must be device memory");
    dem_status st = launch_eval(ctx);
    if (st) return st;
    k_read_contacts<<<nblk(ctx->ncap, 256), 256, 0, ctx->stream>>>(ctx->dev, partner, xi, width);
    CU(cudaGetLastError());
    return DEM_OK;
}

dem_status dem_read_neighbors(dem_ctx* ctx, int32_t* partner, int32_t width, int64_t n)
{
    if (!ctx) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    if (ctx->B != 1) return fail(ctx, DEM_ERR_ARG, "neighbour read-out needs a single-instance context");
    if (dem_status st = refresh_count(ctx)) return st;
    if (n != total_count(ctx) || width < 1 || !partner) return fail(ctx, DEM_ERR_ARG, "bad neighbour arguments");
    if (!is_device_ptr(partner)) return fail(ctx, DEM_ERR_ARG, "neighbour buffer must be device memory");
    dem_status st = launch_rebuild(ctx, ctx->stream);
    if (st) return st;
    k_read_neighbors<<<nblk(ctx->ncap, 256), 256, 0, ctx->stream>>>(ctx->dev, partner, width);
    CU(cudaGetLastError());
    return DEM_OK;
}

dem_status dem_write_contacts(dem_ctx* ctx, const int32_t* partner, const double* xi, int32_t width, int64_t n)
{
    if (!ctx) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    if (ctx->B != 1) return fail(ctx, DEM_ERR_ARG, "contacts I/O needs a single-instance context");
    if (dem_status st = refresh_count(ctx)) return st;
    if (n != total_count(ctx) || width < 1 || !partner || !xi) return fail(ctx, DEM_ERR_ARG, "bad contacts arguments");
    if (!is_device_ptr(partner) || !is_device_ptr(xi)) return fail(ctx, DEM_ERR_ARG, "contacts buffers must be device memory");
    dem_status st = launch_rebuild(ctx, ctx->stream);
    if (st) return st;
    k_write_contacts<<<nblk(ctx->ncap, 256), 256, 0, ctx->stream>>>(ctx->dev, partner, xi, width);
    CU(cudaGetLastError());
    return DEM_OK;
}

dem_status dem_step(dem_ctx* ctx, int64_t nsteps)
{
    NvtxRange nvtx_range("dem_step");
    if (!ctx || nsteps < 0) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    if (!ctx->have_state) return fail(ctx, DEM_ERR_STATE, "write the state before stepping");
    int64_t done = 0;
    while (done < nsteps) {
        if (!ctx->fresh && ctx->gexec && nsteps - done >= ctx->graph_steps) {
            CU(cudaGraphLaunch(ctx->gexec, ctx->stream));
            done += ctx->graph_steps;
            continue;
        }
        dem_status st = launch_rebuild(ctx, ctx->stream);
        if (st) return st;
        st = launch_step(ctx, ctx->fresh ? 1 : 0);
        if (st) return st;
        ctx->fresh = false;
        ++done;
    }
    ctx->steps += nsteps;
    return DEM_OK;
}

dem_status dem_sync_status(dem_ctx* ctx)
{
    if (!ctx) return DEM_ERR_ARG;
    CU(cudaStreamSynchronize(ctx->stream));
    unsigned stv = 0;
    CU(cudaMemcpy(&stv, &ctx->dev.g->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    ctx->status |= stv;
    return check_status(ctx);
}

dem_status dem_instance_info_get(dem_ctx* ctx, int32_t k, dem_instance_info* out)
{
    if (!ctx || !out || k < 0 || k >= ctx->B) return DEM_ERR_ARG;
    const InstC& c = ctx->ic[k];
    const HostInstLo& h = ctx->hl[k];
    out->q = h.q;
    for (int a = 0; a < 3; ++a) {
        out->lo[a] = h.lo[a];
        out->hi[a] = h.lo[a] + (double)c.ext[a] * h.q;
        out->ncell[a] = c.nc[a];
    }
    if (dem_status st = refresh_count(ctx)) return st;
    out->n = ctx->count[k];
    out->capacity = c.cap;
    return DEM_OK;
}

dem_status dem_stats(dem_ctx* ctx, dem_stats_t* out)
{
    if (!ctx || !out) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    memset(out, 0, sizeof(*out));
    out->steps = ctx->steps;
    out->step_threads = ctx->graph_fused ? TILE : step_block(ctx);
    out->step_lanes = ctx->step_lanes;
    out->graph_fused = ctx->graph_fused ? 1 : 0;
    if (dem_status st = refresh_count(ctx)) return st;
    out->particles = total_count(ctx);
    if (!ctx->have_state) return DEM_OK;
    dem_status st = launch_eval(ctx);
    if (st) return st;
    CU(cudaMemsetAsync(&ctx->dev.g->sum_list, 0, 24, ctx->stream));
    k_stats<<<nblk(ctx->ncap, 256), 256, 0, ctx->stream>>>(ctx->dev);
    CU(cudaGetLastError());
    Glob gl;
    CU(cudaMemcpyAsync(&gl, ctx->dev.g, sizeof(Glob), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    out->rebuilds = (int64_t)gl.rebuilds;
    out->list_entries = (int64_t)gl.sum_list;
    out->contacts = (int64_t)gl.sum_contacts;
    out->wall_contacts = (int64_t)gl.sum_wall;
    ctx->status |= gl.status;
    return check_status(ctx);
}

dem_status dem_set_graph(dem_ctx* ctx, int32_t steps_per_graph)
{
    if (!ctx || steps_per_graph < 0 || steps_per_graph > 4096) return DEM_ERR_ARG;
    return build_graph(ctx, steps_per_graph);
}

dem_status dem_set_step_block(dem_ctx* ctx, int32_t threads)
{
    if (!ctx) return DEM_ERR_ARG;
    if (threads != 0 && threads != 64 && threads != 128 && threads != 256 && threads != SMW_BS)
        return fail(ctx, DEM_ERR_ARG, "step block must be 0 (automatic), 64, 128, 256 or 896 threads");
    if (threads == SMW_BS && (ctx->B != 1 || ctx->grid_smw <= 0))
        return fail(ctx, DEM_ERR_STATE, "896-thread (SM-wide) step blocks need a single-instance context");
    if (threads != 0 && threads != 128 && ctx->step_lanes > 1)
        return fail(ctx, DEM_ERR_STATE, "several lanes per particle run at 128 threads per block");
    ctx->step_bs = threads;
    return ctx->graph_steps > 0 ? build_graph(ctx, ctx->graph_steps) : DEM_OK;
}

dem_status dem_set_list_build(dem_ctx* ctx, int32_t staged)
{
    if (!ctx) return DEM_ERR_ARG;
    if (staged != 0 && staged != 1) return fail(ctx, DEM_ERR_ARG, "list build must be 0 (direct scan) or 1 (staged)");
    ctx->list_staged = staged != 0;
    return ctx->graph_steps > 0 ? build_graph(ctx, ctx->graph_steps) : DEM_OK;   // the graph holds the chain
}

dem_status dem_test_stall_barrier(dem_ctx* ctx)
{
    if (!ctx) return DEM_ERR_ARG;
    static const unsigned one = 1u;
    CU(cudaMemcpyAsync(&ctx->dev.g->test_stall, &one, sizeof(unsigned), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

dem_status dem_set_graph_mode(dem_ctx* ctx, int32_t mode)
{
    if (!ctx) return DEM_ERR_ARG;
    if (mode < 0 || mode > 2) return fail(ctx, DEM_ERR_ARG, "graph mode must be 0 (by size), 1 (a kernel per step) or 2 (fused)");
    const int old = ctx->graph_mode;
    ctx->graph_mode = mode;
    if (ctx->graph_steps <= 0) return DEM_OK;
    dem_status st = build_graph(ctx, ctx->graph_steps);
    if (st) {
        ctx->graph_mode = old;                 // keep the previous graph
        const std::string msg = ctx->err;
        dem_status st2 = build_graph(ctx, ctx->graph_steps);
        if (st2) return st2;
        return fail(ctx, st, msg);
    }
    return DEM_OK;
}

dem_status dem_set_step_lanes(dem_ctx* ctx, int32_t lanes)
{
    if (!ctx) return DEM_ERR_ARG;
    if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8)
        return fail(ctx, DEM_ERR_ARG, "lanes per particle must be 0 (by size), 1, 2, 4 or 8");
    if (lanes == 0) {
        // by size: one lane while the rows fill at least half of the resident threads of the
        // one-lane kernel, else the most lanes whose threads are all resident at once
        int nsm = 0, b1 = 0, bl = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_step<0, false, 128>, 128, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, k_step<0, false, 128, 2>, 128, 0);
        cudaGetLastError();
        const long long rows = (long long)ctx->ntiles * TILE;
        const long long r1 = (long long)std::max(1, nsm) * std::max(1, b1) * 128;
        const long long rl = (long long)std::max(1, nsm) * std::max(1, bl) * 128;
        lanes = 1;
        // fused steps (by default when the live tiles' blocks are resident at once): the most
        // lanes whose blocks are all resident
        long long live = 0;
        for (int k = 0; k < ctx->B; ++k) live += 2 * ((ctx->count[k] + 2 * TILE - 1) / (2 * TILE));
        int bf = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_steps<false, 2>, 128, 0);
        cudaGetLastError();
        const long long gf = (long long)std::max(1, nsm) * std::max(1, bf);
        if (ctx->graph_mode != 1 && live <= gf) {
            for (int l = 8; l >= 2; l >>= 1)
                if ((long long)l * live <= gf) {
                    lanes = l;
                    break;
                }
        } else if (2 * rows < r1) {
            for (int l = 8; l >= 2; l >>= 1)
                if ((long long)l * rows <= rl) {
                    lanes = l;
                    break;
                }
        }
        if (ctx->step_bs != 0 && ctx->step_bs != 128) lanes = 1;
    }
    if (lanes > 1 && ctx->step_bs != 0 && ctx->step_bs != 128)
        return fail(ctx, DEM_ERR_STATE, "several lanes per particle run at 128 threads per block");
    ctx->step_lanes = lanes;
    return ctx->graph_steps > 0 ? build_graph(ctx, ctx->graph_steps) : DEM_OK;
}

dem_status dem_graph_step_kernel_ms(dem_ctx* ctx, double* total_ms, int32_t* count)
{
    if (!ctx || !total_ms || !count) return DEM_ERR_ARG;
    if (!ctx->gexec) return fail(ctx, DEM_ERR_STATE, "no step graph has been built");
    CU(cudaStreamSynchronize(ctx->stream));
    double t = 0.0;
    for (size_t i = 0; i < ctx->ev0.size(); ++i) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, ctx->ev0[i], ctx->ev1[i]));
        t += ms;
    }
    *total_ms = t;
    *count = ctx->graph_fused ? (int32_t)ctx->graph_steps : (int32_t)ctx->ev0.size();
    return DEM_OK;
}

dem_status dem_grid_fields(dem_ctx* ctx, int32_t k, const double lo[3], double h, const int32_t n[3], double* out,
                           int64_t out_len)
{
    if (!ctx || !lo || !n || !out) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    if (k < 0 || k >= ctx->B) return fail(ctx, DEM_ERR_ARG, "no such instance");
    if (!(h > 0.0) || n[0] < 1 || n[1] < 1 || n[2] < 1) return fail(ctx, DEM_ERR_ARG, "empty grid");
    const long long ncell = (long long)n[0] * n[1] * n[2];
    if (out_len != 5 * ncell) return fail(ctx, DEM_ERR_ARG, "out must hold 5 values per cell");
    if (!is_device_ptr(out)) return fail(ctx, DEM_ERR_ARG, "out must be device memory");
    if (!ctx->have_state) return fail(ctx, DEM_ERR_STATE, "write the state first");
    dem_status st = launch_eval(ctx);
    if (st) return st;
    CU(cudaMemsetAsync(out, 0, sizeof(double) * 5 * ncell, ctx->stream));
    k_grid_sums<<<ctx->grid_rb, 256, 0, ctx->stream>>>(ctx->dev, k, ctx->d_hl, lo[0], lo[1], lo[2], h, n[0], n[1],
                                                       n[2], out);
    CU(cudaGetLastError());
    k_grid_finish<<<nblk(ncell, 256) > 4096 ? 4096 : nblk(ncell, 256), 256, 0, ctx->stream>>>(out, ncell, h * h * h);
    CU(cudaGetLastError());
    return DEM_OK;
}

const char* dem_last_error(const dem_ctx* ctx)
{
    if (!ctx) return g_cfg_err.c_str();
    return ctx->err.c_str();
}

}  // extern "C"

// ================================================================ rollout (host)

namespace {

size_t snap_layout(const dem_ctx* ctx, Layout& L, Snap* S, char* base)
{
    const size_t N = (size_t)ctx->ncap, Lm = (size_t)ctx->Lmax;
    size_t o_pos = L.take(N * 16), o_vel = L.take(N * 16), o_omg = L.take(N * 16), o_h = L.take(N * Lm * 12),
           o_hm = L.take(N * 4), o_wh = L.take(N * 16), o_disp = L.take(sizeof(float) * ctx->B);
    if (S && base) {
        S->pos = (int4*)(base + o_pos);
        S->vel = (float4*)(base + o_vel);
        S->omg = (float4*)(base + o_omg);
        S->hist = (float*)(base + o_h);
        S->hmask = (unsigned*)(base + o_hm);
        S->whist = (float4*)(base + o_wh);
        S->disp = (float*)(base + o_disp);
    }
    return L.total;
}

size_t rollout_layout(dem_ctx* ctx, long long nsteps, long long K, char* base)
{
    Layout L;
    const int ncp = (int)((nsteps + K - 1) / K) + 1;
    const int nseg = (int)std::min<long long>(K, nsteps);
    if (base) {
        ctx->ro.ck.assign(ncp, Snap{});
        ctx->ro.seg.assign(nseg, Snap{});
    }
    for (int i = 0; i < ncp; ++i) snap_layout(ctx, L, base ? &ctx->ro.ck[i] : nullptr, base);
    for (int i = 0; i < nseg; ++i) snap_layout(ctx, L, base ? &ctx->ro.seg[i] : nullptr, base);
    const size_t N = (size_t)ctx->ncap, Lm = (size_t)ctx->Lmax;
    size_t o_xb = L.take(N * 16), o_vb = L.take(N * 16), o_wb = L.take(N * 16), o_Fb = L.take(N * 16),
           o_Tb = L.take(N * 16), o_xib = L.take(N * Lm * 12), o_wxib = L.take(N * 16), o_thb = L.take(N * 24);
    if (base) {
        AdjBufs& a = ctx->ro.a;
        a.xb = (float4*)(base + o_xb);
        a.vb = (float4*)(base + o_vb);
        a.wb = (float4*)(base + o_wb);
        a.Fb = (float4*)(base + o_Fb);
        a.Tb = (float4*)(base + o_Tb);
        a.xib = (float*)(base + o_xib);
        a.wxib = (float4*)(base + o_wxib);
        a.thb = (double*)(base + o_thb);
    }
    return L.total;
}

dem_status set_frozen(dem_ctx* ctx, unsigned v)
{
    CU(cudaMemcpyAsync(&ctx->dev.g->frozen, &v, sizeof(unsigned), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

dem_status snap(dem_ctx* ctx, const Snap& S, bool save)
{
    if (save) k_snap<true><<<ctx->grid_rb, TILE, 0, ctx->stream>>>(ctx->dev, S);
    else k_snap<false><<<ctx->grid_rb, TILE, 0, ctx->stream>>>(ctx->dev, S);
    CU(cudaGetLastError());
    return DEM_OK;
}

dem_status step_once(dem_ctx* ctx, int prime)
{
    if (dem_status st = launch_step(ctx, prime)) return st;   // rollouts refuse walls
    CU(cudaGetLastError());
    return DEM_OK;
}

dem_status upload_material(dem_ctx* ctx)
{
    CU(cudaMemcpyAsync((void*)ctx->dev.ic, ctx->ic.data(), sizeof(InstC) * ctx->B, cudaMemcpyHostToDevice,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

}  // namespace

extern "C" {

dem_status dem_set_material(dem_ctx* ctx, const double* params)
{
    if (!ctx || !params) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    for (int k = 0; k < ctx->B; ++k) {
        const double E = params[3 * k], e = params[3 * k + 1], mu = params[3 * k + 2];
        if (!(E > 0) || !(e > 0 && e <= 1) || !(mu >= 0)) return fail(ctx, DEM_ERR_ARG, "need E > 0, 0 < e <= 1, mu >= 0");
        InstC& c = ctx->ic[k];
        const double nu = ctx->nu[k];
        const double Eeff = 1.0 / (2.0 * (1.0 - nu * nu) / E);
        const double Geff = 1.0 / (2.0 * 2.0 * (2.0 - nu) * (1.0 + nu) / E);
        const double le = std::log(e);
        c.c_kn = (float)(4.0 / 3.0 * Eeff);
        c.c_kt = (float)(8.0 * Geff);
        c.nbeta = (float)(-(le / std::sqrt(le * le + M_PI * M_PI)));
        c.mu = (float)mu;
        if (c.mu_w_follows) c.mu_w = (float)mu;
        c.inv_E = (float)(1.0 / E);
        c.dnb_de = (float)(-(M_PI * M_PI) / (e * std::pow(le * le + M_PI * M_PI, 1.5)));
    }
    return upload_material(ctx);
}

dem_status dem_set_walls(dem_ctx* ctx, int32_t k, const double* axis, int32_t npts, const double* points,
                         double z_remove)
{
    if (!ctx) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    if (k < 0 || k >= ctx->B) return fail(ctx, DEM_ERR_ARG, "instance index out of range");
    if (npts != 0 && (npts < 2 || npts > MAX_WP || !points || !axis))
        return fail(ctx, DEM_ERR_ARG, "need 0 or 2 .. 8 polyline points and the axis");
    InstC& c = ctx->ic[k];
    const HostInstLo& h = ctx->hl[k];
    const double q = h.q;
    InstC w = c;
    WallGeo wg{};
    w.nwp = npts;
    w.wmag = 0.f;
    if (npts) {
        if (!(std::isfinite(axis[0]) && std::isfinite(axis[1]))) return fail(ctx, DEM_ERR_ARG, "axis must be finite");
        w.wax = (axis[0] - h.lo[0]) / q;
        w.way = (axis[1] - h.lo[1]) / q;
        if (!(std::fabs(w.wax) < 1.0e9 && std::fabs(w.way) < 1.0e9)) return fail(ctx, DEM_ERR_ARG, "axis far outside the box");
        w.waxi = (int)std::floor(w.wax);
        w.wayi = (int)std::floor(w.way);
        w.waxf = (float)(w.wax - w.waxi);
        w.wayf = (float)(w.way - w.wayi);
        double mag = 0.0;
        for (int i = 0; i < npts; ++i) {
            const double rho = points[2 * i], z = points[2 * i + 1];
            if (!(std::isfinite(rho) && std::isfinite(z) && rho >= 0.0)) return fail(ctx, DEM_ERR_ARG, "polyline points need rho >= 0, finite z");
            w.wp[2 * i] = rho / q;
            w.wp[2 * i + 1] = (z - h.lo[2]) / q;
            if (!(w.wp[2 * i] < 2.0e9 && std::fabs(w.wp[2 * i + 1]) < 2.0e9)) return fail(ctx, DEM_ERR_ARG, "polyline far outside the box");
            w.wpf[2 * i] = (float)w.wp[2 * i];
            w.wpf[2 * i + 1] = (float)w.wp[2 * i + 1];
            mag = std::max(mag, std::max(w.wp[2 * i], std::fabs(w.wp[2 * i + 1])));
            if (i > 0 && points[2 * i] == points[2 * i - 2] && points[2 * i + 1] == points[2 * i - 1])
                return fail(ctx, DEM_ERR_ARG, "polyline segments need a non-zero length");
        }
        for (int i = 0; i + 1 < npts; ++i) {
            const double dr = w.wp[2 * i + 2] - w.wp[2 * i], dz = w.wp[2 * i + 3] - w.wp[2 * i + 1];
            const double len = std::sqrt(dr * dr + dz * dz);
            wg.ur[i] = dr / len;
            wg.uz[i] = dz / len;
            wg.len[i] = len;
            const float drf = w.wpf[2 * i + 2] - w.wpf[2 * i], dzf = w.wpf[2 * i + 3] - w.wpf[2 * i + 1];
            wg.inv2[i] = 1.0f / (drf * drf + dzf * dzf);
        }
        w.wmag = (float)mag;
    }
    w.zrem = INT_MIN;
    if (std::isnan(z_remove)) return fail(ctx, DEM_ERR_ARG, "z_remove is NaN");
    if (z_remove > -INFINITY) {
        const double zu = std::ceil((z_remove - h.lo[2]) / q);   // removed: z < z_remove, i.e. z_units < zu
        if (!(zu < 2.0e9)) return fail(ctx, DEM_ERR_ARG, "z_remove above the representable range");
        if (zu > -2.0e9) w.zrem = (int)zu;
    }
    c = w;
    bool any = false;
    for (int i = 0; i < ctx->B; ++i) any |= ctx->ic[i].nwp >= 2;
    const bool rebuild_graph = any != ctx->walls && ctx->gexec;
    ctx->walls = any;
    // the wall-contact history of the instance starts empty
    const size_t n = (size_t)c.cap, ncap = (size_t)ctx->dev.ncap;
    for (int b = 0; b < 2; ++b)
        for (int half = 0; half < 2; ++half)
            CU(cudaMemsetAsync(ctx->dev.wseg[b] + half * ncap + c.slot0, 0, n * sizeof(float4), ctx->stream));
    CU(cudaMemcpyAsync((void*)(ctx->dev.wgeo + k), &wg, sizeof(WallGeo), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));                        // wg is a local
    if (dem_status st = upload_material(ctx)) return st;
    return rebuild_graph ? build_graph(ctx, ctx->graph_steps) : DEM_OK;
}

dem_status dem_wall_removed(dem_ctx* ctx, int32_t k, double* out)
{
    if (!ctx || !out) return DEM_ERR_ARG;
    if (k < 0 || k >= ctx->B) return fail(ctx, DEM_ERR_ARG, "instance index out of range");
    CU(cudaMemcpyAsync(out, ctx->dev.wrem + 2 * k, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return check_status(ctx);
}

dem_status dem_rollout_workspace(dem_ctx* ctx, int64_t nsteps, int64_t checkpoint_every, int64_t* bytes)
{
    if (!ctx || !bytes || nsteps < 1 || checkpoint_every < 1) return DEM_ERR_ARG;
    *bytes = (int64_t)rollout_layout(ctx, nsteps, checkpoint_every, nullptr);
    return DEM_OK;
}

dem_status dem_rollout_forward(dem_ctx* ctx, int64_t nsteps, int64_t checkpoint_every, void* ws, int64_t ws_bytes)
{
    NvtxRange nvtx_range("dem_rollout_forward");
    if (!ctx || nsteps < 1 || checkpoint_every < 1 || !ws) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    if (!ctx->have_state) return fail(ctx, DEM_ERR_STATE, "write the state before a rollout");
    for (int k = 0; k < ctx->B; ++k)
        if (ctx->ic[k].nwp || ctx->ic[k].zrem != INT_MIN)
            return fail(ctx, DEM_ERR_STATE, "rollouts do not differentiate axisymmetric walls or removal");
    const size_t need = rollout_layout(ctx, nsteps, checkpoint_every, nullptr);
    if ((size_t)ws_bytes < need || ((uintptr_t)ws & 255)) return fail(ctx, DEM_ERR_ARG, "rollout workspace too small");
    rollout_layout(ctx, nsteps, checkpoint_every, (char*)ws);
    Rollout& ro = ctx->ro;
    ro.nsteps = nsteps;
    ro.K = checkpoint_every;
    ro.ncp = (int)ro.ck.size();
    ro.prime0 = ctx->fresh;
    dem_status st = launch_rebuild(ctx, ctx->stream);       // the lists the whole rollout uses
    if (st) return st;
    if ((st = set_frozen(ctx, 1u))) return st;
    for (long long s = 0; s < nsteps; ++s) {
        if (s % ro.K == 0 && (st = snap(ctx, ro.ck[s / ro.K], true))) return st;
        if ((st = step_once(ctx, (s == 0 && ro.prime0) ? 1 : 0))) return st;
    }
    if ((st = snap(ctx, ro.ck[ro.ncp - 1], true))) return st;
    if ((st = set_frozen(ctx, 0u))) return st;
    ctx->fresh = false;
    ctx->steps += nsteps;
    ro.ready = true;
    return dem_sync_status(ctx);
}

dem_status dem_observables(dem_ctx* ctx, const double* axis, double* out)
{
    if (!ctx || !axis || !out) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    if (!ctx->have_state) return fail(ctx, DEM_ERR_STATE, "write the state first");
    dem_status st = launch_eval(ctx);
    if (st) return st;
    std::vector<double> sm(16 * ctx->B, 0.0);
    for (int k = 0; k < ctx->B; ++k) { sm[16 * k] = axis[2 * k]; sm[16 * k + 1] = axis[2 * k + 1]; }
    CU(cudaMemcpyAsync(ctx->dev.small, sm.data(), sizeof(double) * sm.size(), cudaMemcpyHostToDevice, ctx->stream));
    k_obs<<<ctx->B, 256, 0, ctx->stream>>>(ctx->dev, ctx->d_hl);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(sm.data(), ctx->dev.small, sizeof(double) * sm.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < ctx->B; ++k) { out[2 * k] = sm[16 * k + 2]; out[2 * k + 1] = sm[16 * k + 3]; }
    return dem_sync_status(ctx);
}

dem_status dem_rollout_adjoint(dem_ctx* ctx, const double* weights, const double* axis, double* grad)
{
    NvtxRange nvtx_range("dem_rollout_adjoint");
    if (!ctx || !weights || !axis || !grad) return DEM_ERR_ARG;
    if (ctx->status) return check_status(ctx);
    Rollout& ro = ctx->ro;
    if (!ro.ready) return fail(ctx, DEM_ERR_STATE, "run dem_rollout_forward first");
    cudaStream_t s = ctx->stream;
    // observables and their seeds at the final step N
    dem_status st = launch_eval(ctx);
    if (st) return st;
    std::vector<double> sm(16 * ctx->B, 0.0);
    for (int k = 0; k < ctx->B; ++k) {
        sm[16 * k] = axis[2 * k];
        sm[16 * k + 1] = axis[2 * k + 1];
        sm[16 * k + 5] = weights[2 * k];
        sm[16 * k + 6] = weights[2 * k + 1];
    }
    CU(cudaMemcpyAsync(ctx->dev.small, sm.data(), sizeof(double) * sm.size(), cudaMemcpyHostToDevice, s));
    k_obs<<<ctx->B, 256, 0, s>>>(ctx->dev, ctx->d_hl);
    k_adj_seed<<<ctx->grid_rb, TILE, 0, s>>>(ctx->dev, ro.a, ctx->d_hl);
    CU(cudaGetLastError());
    if ((st = set_frozen(ctx, 1u))) return st;
    const long long N = ro.nsteps, K = ro.K;
    // v^N = v^{N-1/2} + dt/2 F^N / m: the evaluation at N with a half kick and no drift
    k_adj_prep<<<ctx->grid_rb, TILE, 0, s>>>(ctx->dev, ro.a, 0.5f, 0);
    k_adj_force<<<ctx->grid_rb, TILE, 0, s>>>(ctx->dev, ro.a, ro.ck[ro.ncp - 1], 0);
    CU(cudaGetLastError());
    for (int c = ro.ncp - 2; c >= 0; --c) {
        const long long s0 = (long long)c * K, s1 = std::min(s0 + K, N);
        if ((st = snap(ctx, ro.ck[c], false))) return st;          // restore step s0
        for (long long t = s0; t < s1; ++t) {                      // recompute the segment
            if ((st = snap(ctx, ro.seg[t - s0], true))) return st;
            if ((st = step_once(ctx, (t == 0 && ro.prime0) ? 1 : 0))) return st;
        }
        for (long long t = s1 - 1; t >= s0; --t) {
            const bool pr = t == 0 && ro.prime0;
            k_adj_prep<<<ctx->grid_rb, TILE, 0, s>>>(ctx->dev, ro.a, pr ? 0.5f : 1.0f, 1);
            k_adj_force<<<ctx->grid_rb, TILE, 0, s>>>(ctx->dev, ro.a, ro.seg[t - s0], pr ? 1 : 0);
            CU(cudaGetLastError());
        }
    }
    k_adj_reduce<<<ctx->B, 256, 0, s>>>(ctx->dev, ro.a);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(sm.data(), ctx->dev.small, sizeof(double) * sm.size(), cudaMemcpyDeviceToHost, s));
    if ((st = snap(ctx, ro.ck[ro.ncp - 1], false))) return st;    // back to the final state
    if ((st = set_frozen(ctx, 0u))) return st;
    for (int k = 0; k < ctx->B; ++k)
        for (int q = 0; q < 3; ++q) grad[3 * k + q] = sm[16 * k + 8 + q];
    return dem_sync_status(ctx);
}

}  // extern "C"
