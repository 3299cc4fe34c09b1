/*
 * Shared declarations of the FP64 oracle (test infrastructure only; see
 * dem_oracle.c).  Parameter block P (flat array of doubles):
 *   0 E   1 nu   2 e   3 mu   4 mu_wall   5 dt   6..8 g   9..11 lo
 *   12..14 hi   15..17 periodic flags   18 floor_on   19 floor_z
 *   20..22 floor velocity   23 clamp_fn (1: no tensile normal force)
 *   24 number of wall profile points (0: no walls)   25..26 wall axis (x, y)
 *   27..42 up to 8 profile points (rho, z) of the axisymmetric walls
 */
#ifndef DEM_ORACLE_COMMON_H
#define DEM_ORACLE_COMMON_H
#include <stdint.h>

#define P_E 0
#define P_NU 1
#define P_REST 2
#define P_MU 3
#define P_MUW 4
#define P_DT 5
#define P_G 6
#define P_LO 9
#define P_HI 12
#define P_PER 15
#define P_FLOOR 18
#define P_FLOORZ 19
#define P_FLOORV 20
#define P_CLAMP 23
#define P_NWP 24
#define P_WAX 25
#define P_WAY 26
#define P_WP 27
#define ORC_MAXWP 8

#define ORC_PI 3.14159265358979323846

typedef struct { int64_t i, j; } pair_t;

/* index pairs i < j with |x_ij| < r_i + r_j + extra (malloc'd, sorted by (i, j)) */
pair_t *orc_find_pairs(const double *P, int64_t n, const double *x, const double *r, double extra,
                       int use_cells, int64_t *out_cnt);

#endif
