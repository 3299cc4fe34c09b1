// Internal layout shared by the library's translation units (never by the oracle).
//
// Device data of a context (all carved from the caller's workspace):
//   slots      particles of instance k live in slots [slot0_k, slot0_k + n_k);
//              slot0_k is a multiple of TILE so that a thread block of the step
//              kernel never straddles two instances.
//   state      double-buffered SoA, 48 B per particle:
//                pos int4   {x, y, z, r}  32-bit fixed point, units of q
//                vel float4 {vx, vy, vz, id | floor-contact bit 31}
//                omg float4 {wx, wy, wz, m}
//              buffer cur_k holds step n, the step kernel writes cur_k ^ 1.
//   lists      double-buffered (parity lp_k), entry-major for coalescing:
//                nbr  int32 [Lmax][ncap]      slot of the e-th neighbour
//                hist float  [3][Lmax][ncap]  tangential overlap of entry e,
//                                             seen from the row's particle (the
//                                             partner's row holds its negative)
//                hmask u32  [ncap]            bit e set: entry e holds a non-zero
//                                             overlap (the contact was active)
//                cnt  int32 [ncap]            row length; rows are ordered by
//                                             d^2 - (r_i + r_j)^2 at the build,
//                                             then by neighbour ID
//                whist float4 [ncap]          floor-contact tangential overlap
//                wseg  float4 [2][ncap]       up to two axisymmetric-wall contacts:
//                                             {xi, segment + 1 (bits); 0: empty}
//   cells      per instance a Morton-ordered code range [code0_k, code0_k + ncode_k)
//              with counts and exclusive starts, rebuilt with the lists.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cgdem {

constexpr int TILE = 128;      // step-kernel block size = slot alignment of an instance
constexpr int MAXL = 32;       // largest list width (one bit per entry in a 32-bit mask)
constexpr unsigned ID_MASK = 0x3fffffffu;   // particle ID (< 2^30)
constexpr unsigned GONE_BIT = 0x40000000u;  // removed: dropped at the next list build
constexpr unsigned WALL_BIT = 0x80000000u;  // in contact with the floor at the last step
constexpr int MAX_WP = 8;      // points of an axisymmetric wall polyline

// Axisymmetric walls: the offsets (a, b) = (rho, z) - nearest point of wall segment k of an
// instance (the segment from polyline point k to point k + 1, in the (rho, z) half-plane of
// the particle); lengths in units of q from the box origin.
struct InstC;
__device__ __forceinline__ void wall_seg_offset(const InstC& c, int k, double rho, double z, double& a, double& b);

// device status bits
constexpr unsigned ST_CAPACITY = 1u;
constexpr unsigned ST_NONFINITE = 2u;
constexpr unsigned ST_ESCAPED = 4u;
constexpr unsigned ST_TIMEOUT = 8u;
constexpr unsigned ST_TRUNC = 16u;
constexpr unsigned ST_SKIN = 32u;     // displacement exceeded the skin while lists were frozen
constexpr unsigned ST_INSERT = 64u;   // coupling insertions beyond the fine level's capacity (not appended)
constexpr unsigned ST_BOUNDS = 128u;  // DEM_CHECKS builds: an index out of range (the access skipped)

// Bounds-checked builds (-DDEM_CHECKS=1): the step kernel's gathered particle indices (touch and
// contact passes) and the list build's cell codes and candidate ranges are tested against the
// capacity before use; a violation sets ST_BOUNDS and the access is replaced by a harmless one.
// (The coupling kernels walk slots directly and clamp every cell index they compute.)  Off by
// default: the checks cost issue slots.
#ifndef DEM_CHECKS
#define DEM_CHECKS 0
#endif

// constant description of one instance (host-computed at create)
struct InstC {
    int slot0, cap;
    int ext[3];          // box extent per axis in units of q
    int per[3];          // periodic flags
    int half[3];         // ext / 2 on periodic axes
    int nc[3];           // cells per axis
    int spread_off[3];   // offsets of the per-axis Morton spread tables
    int code0, ncode;
    int floor_on;
    int skin;            // skin in units
    int clamp_fn;
    int mu_w_follows;    // 1: the wall friction is mu (it follows mu in derivatives)
    float q, dt, dt_over_q, skin_f;
    float g[3];
    float floor_v[3];
    float c_kn, c_kt, nbeta, mu, mu_w;   // 4/3 E_eff, 8 G_eff, -beta, mu, mu_wall
    float gt_ratio;                      // gamma_t / gamma_n = sqrt(2 c_kt / (3 c_kn))
    float inv_E;                         // 1 / E (c_kn and c_kt are proportional to E)
    float dnb_de;                        // d(-beta)/de
    // axisymmetric walls: the surface of revolution of the polyline (rho_i, z_i) about the
    // vertical axis (wax, way); lengths in units of q from the box origin
    int nwp;                             // polyline points (0: no walls)
    int zrem;                            // particles whose centre falls below z = zrem are removed
                                         // (INT_MIN: none)
    int waxi, wayi;                      // axis: whole units and fraction (float pre-test, direction)
    float waxf, wayf;
    float wmag;                          // largest polyline coordinate (float pre-test tolerance)
    double wax, way;
    double wp[2 * MAX_WP];
    float wpf[2 * MAX_WP];
};
static_assert(sizeof(InstC) <= 4 * TILE, "the step kernel stages InstC in shared memory, one word per thread");

// per-segment constants of an instance's axisymmetric walls (outside InstC, which every step
// block stages: the plain step kernel does not pay for them)
struct WallGeo {
    double ur[MAX_WP], uz[MAX_WP];       // unit tangent (rho, z) of segment k (from point k to k + 1)
    double len[MAX_WP];                  // length of segment k [units]
    float inv2[MAX_WP];                  // 1 / |segment k|^2 from the float points (float pre-test)
};

__device__ __forceinline__ void wall_seg_offset(const InstC& c, int k, double rho, double z, double& a, double& b)
{
    const double r0 = c.wp[2 * k], z0 = c.wp[2 * k + 1];
    const double dr = c.wp[2 * k + 2] - r0, dz = c.wp[2 * k + 3] - z0;
    const double t = fmin(fmax(((rho - r0) * dr + (z - z0) * dz) / (dr * dr + dz * dz), 0.0), 1.0);
    a = rho - (r0 + t * dr);
    b = z - (z0 + t * dz);
}

// dynamic state of one instance (device-resident)
struct InstD {
    int n;               // live particles (slots slot0 .. slot0 + n - 1)
    int cur;             // state buffer holding the current step
    int lp;              // list buffer parity
    int flag;            // 0 none, 1 rebuild pending, 2 rebuild with cleared history
    float disp;          // accumulated per-step displacement bound since the last build [units]
    unsigned stepmax;    // this step's largest displacement (float bits)
    int nid;             // IDs handed out so far (n plus removed particles); IDs are never reused
    int n_new;           // live particles after the pending rebuild (removed ones dropped)
    int fext;            // 1: add the per-particle external force fext to the contact forces
    int nbin;            // slots below slot0 + nbin are in the cell lists of the last build
    int pad[2];
};

struct Glob {
    unsigned status;
    unsigned any;              // some instance has flag != 0
    unsigned counter;          // last-block detection of the step kernel
    unsigned frozen;           // 1: lists are frozen (differentiable rollout), no rebuilds
    unsigned long long rebuilds;
    unsigned long long sum_list;
    unsigned long long sum_contacts;
    unsigned long long sum_wall;
    long long err_slot;
    long long err_val;         // DEM_CHECKS builds: the index found out of range, and where
    int err_site;              // (1 cell code, 2 cell range of the list build; 3 touch pass,
    int err_pad;               //  4 contact pass of the step kernel)
    unsigned bar_gen;          // fused steps: grid-barrier generation (bumped by each release)
    unsigned bar_pad;
    long long remain;          // fused steps: steps still to do in the current graph launch
    int nlive;                 // entries of live_tiles
    unsigned test_stall;       // 1: the next fused launch's first block skips its first barrier
    unsigned pool;             // SM-wide step blocks: slices claimed from the shared pool this launch
};

// kernel-visible pointers of a context
struct Dev {
    int4* pos[2];
    float4* vel[2];
    float4* omg[2];
    int* nbr[2];
    float* hist[2];
    int* cnt[2];
    unsigned* hmask[2];        // bit e: entry e holds a non-zero tangential overlap
    float4* fext[2];           // external force per particle (coupling controllers), list parity
    float4* whist[2];
    float4* wseg[2];           // [2][ncap] axisymmetric-wall contacts, list parity
    double* wrem;              // [2 * B] particles and mass removed below the removal height
    unsigned* cellcode;
    unsigned* cslot;
    int* perm;                 // cell-order position -> old slot
    int* fin;                  // cell-order position -> new slot (tiles reordered by contact count)
    int4* spos;                // positions in cell order (list build)
    int* sid;                  // particle IDs in cell order (list build)
    unsigned* ccount;
    uint2* crange;             // per cell code: {first cell-order position (exclusive scan), count}
    unsigned* part;
    int* part_inst;            // instance owning each scan chunk of cell codes (-1: padding)
    int* slot_of_id;
    int* tile_inst;
    const WallGeo* wgeo;       // [B] wall segment constants
    int* live_tiles;           // the tiles fused steps walk: each instance's first tiles holding its
                               // live slots, in whole pairs (g->nlive of them; set by each list build)
    const InstC* ic;
    InstD* id;
    const unsigned* spread;
    Glob* g;
    long long* goff;           // [B+1] global offsets of instances in user arrays
    float4* outF;
    float4* outT;
    float4* outV;
    float4* outW;
    float4* outWX;             // floor-contact xi at the evaluated step
    float* xi_out;             // [3][Lmax][ncap]
    unsigned long long* cmask; // contact bits per list entry at the evaluated step
    double* stage;             // [3 * ncap] staging for host transfers
    double* small;             // [16 * B] per-instance scratch of observables and gradients
    int ncap;
    int ntiles;
    int B;
    int Lmax;
    unsigned ncodes;
    unsigned nparts;
};

// DEM_CHECKS: true if i lies in [0, n); otherwise records ST_BOUNDS, the slot s, the index and
// the check's site
__device__ __forceinline__ bool in_range(const Dev& d, long long i, long long n, int s, int site)
{
    if (!DEM_CHECKS || (i >= 0 && i < n)) return true;
    atomicOr(&d.g->status, ST_BOUNDS);
    d.g->err_slot = s;
    d.g->err_val = i;
    d.g->err_site = site;
    return false;
}

// host-side description of an instance's frame (origin, quantum, density)
struct HostInstLo {
    double lo[3];
    double q;
    double rho;
};

// snapshot of the dynamic state of a context (differentiable rollouts)
struct Snap {
    int4* pos;
    float4* vel;
    float4* omg;
    float* hist;
    unsigned* hmask;
    float4* whist;
    float* disp;       // per instance: displacement bound accumulated since the list build
};

// adjoint buffers of a differentiable rollout
struct AdjBufs {
    float4* xb;        // adjoint of x^n [1/m units of the objective]
    float4* vb;        // adjoint of v^{n-1/2}
    float4* wb;        // adjoint of w^{n-1/2}
    float4* Fb;        // adjoint of F^n
    float4* Tb;        // adjoint of T^n
    float* xib;        // adjoint of the stored overlaps, [3][Lmax][ncap], from each row's side
    float4* wxib;      // adjoint of the floor overlap
    double* thb;       // per slot: accumulated d/dE, d/de, d/dmu
};

__device__ __forceinline__ int axis_cell(const InstC& c, int a, int x)
{
    if (x <= 0) return 0;
    long long t = (long long)x * c.nc[a] / c.ext[a];
    return t >= c.nc[a] ? c.nc[a] - 1 : (int)t;
}

__device__ __forceinline__ unsigned cell_code(const Dev& d, const InstC& c, int cx, int cy, int cz)
{
    return (unsigned)c.code0 + d.spread[c.spread_off[0] + cx] + d.spread[c.spread_off[1] + cy] +
           d.spread[c.spread_off[2] + cz];
}

__device__ __forceinline__ int min_image(int dx, int per, int L, int half)
{
    if (per) {
        if (dx > half) dx -= L;
        else if (dx < -half) dx += L;
    }
    return dx;
}

}  // namespace cgdem
