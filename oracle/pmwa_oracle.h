/*
 * pmwa_oracle.h -- plain, slow CPU oracle of the PMWA Monte Carlo sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The GPU
 * product path (paper_1307_0328_gb300/, include/pmwa.h) shares no code,
 * header, table or constant generator with it.
 *
 * What it computes (Masaki-Kato, Suzuki, Harada, Todo, Kawashima,
 * "Parallelized Quantum Monte Carlo Algorithm with Nonlocal Worm Updates"):
 *   - the directed-loop worldline configuration of H_eta = H - eta Q for the
 *     hard-core Bose-Hubbard model (Eq. 5, read as -t sum(b+_i b_j + h.c.)
 *     + V sum n_i n_j - mu sum n_i, written per bond);
 *   - one MC step = Step 1 (temporal-boundary update, Eq. 3, with N_beta > 1
 *     temporal domains) and Step 2 (spatial-boundary update, Eq. 4) every K
 *     sweeps, Step 3 (vertex phase), Step 4 (worm creation, Eq. 1), Step 5 x
 *     N_cycle (worm scattering, Eq. 2), Step 6 (measurement, Supplement S-I);
 *   - the Supplement S-I estimators, resolved by the component of Q, at
 *     arbitrary times and with several points on one interval;
 *   - the on-the-fly vertex generation the paper names as an extension (the
 *     vertex phase confined to windows around the worms), oracle only;
 *   - everything in the fixed deterministic arithmetic that the GPU path also
 *     implements (Philox4x32-10 streams, ziggurat exponentials, fixed-point
 *     time, integer thresholds), so the two can be compared bit for bit.
 *
 * Parity pins: every function here is pinned by tests in tests/test_oracle_*.py
 * against closed forms, exact diagonalisation and invariants (see the test
 * docstrings).  No expected value in the tests comes from the GPU path.
 */
#ifndef PMWA_ORACLE_H
#define PMWA_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t  Lx, Ly;          /* periodic square lattice, both >= 2             */
  double   beta, t, V, mu, eta;
  uint64_t seed;            /* Philox key                                     */
  int32_t  dom_x, dom_y;    /* sites per domain along x / y (divide Lx / Ly)  */
  int32_t  exchange_every;  /* K: Step 2 when sweep % K == 0                  */
  int32_t  n_cycle;         /* Step-5 passes per sweep                        */
  int32_t  sub_block;       /* shifted sub-block edge B (even), 0 = domain    */
  int32_t  init;            /* 0: empty lattice, 1: random half filling,
                               2: checkerboard (x + y even occupied)           */
  uint64_t init_seed;
  double   c_off;           /* vertex-density offset; < 0 means t/2           */
  uint32_t replica;         /* replica id mixed into every Philox counter     */
  int32_t  dom_tau;         /* temporal domains N_beta (1..64): Step 1        */
  double   vertex_window;   /* on-the-fly vertex generation: 0 = off, else the
                               vertex phase of a bond only within this fraction
                               of beta of a worm on its sites (0 < w <= 1)   */
} or_params;

/* One row per measured sweep (Step 6). */
typedef struct {
  uint64_t sweep;
  uint64_t n_v;       /* vertices (diagonal + kinks, all bonds)               */
  uint64_t n_k;       /* kinks                                                */
  uint64_t n_w;       /* worms                                                */
  uint64_t occ_lo;    /* sum_i of occupied imaginary time, in units          */
  uint64_t occ_hi;    /*   beta / 2^62, as a 128-bit integer                  */
  double   q_impr;    /* sum over intervals of x g_sigma(x), x = I eta        */
  uint32_t w_dom_min; /* fewest worms in one domain                           */
  uint32_t dom_empty; /* domains without a worm                               */
} or_row;

typedef struct or_handle or_handle;

/* status codes (same meanings as the product's) */
#define OR_OK        0
#define OR_EINVAL    1
#define OR_ETIMEOUT  3
#define OR_EINVARIANT 5

int   or_create(const or_params* p, or_handle** out);
void  or_destroy(or_handle* h);
int   or_sweep(or_handle* h, int64_t n);            /* full MC steps          */
/* single steps, for fine-grained parity debugging */
int   or_temporal(or_handle* h);                    /* Step 1 (temporal boundaries, Eq. 3) */
int   or_boundary(or_handle* h);                    /* Step 2 (+ Step 3 on boundary bonds) */
int   or_tile(or_handle* h, int stop_after);        /* Steps 3..6, stop_after in {3,4,5,6} */
int   or_check(or_handle* h);                       /* invariants, OR_OK or OR_EINVARIANT   */
int64_t or_rows(or_handle* h, or_row* out, int64_t max_rows); /* drain measured rows  */
/* canonical configuration: u64 n_sites, then per site u64 header
   (count | base_state << 63) followed by count u64 event keys.          */
size_t or_export_bytes(or_handle* h);
int   or_export(or_handle* h, void* buf, size_t bytes);
int   or_import(or_handle* h, const void* buf, size_t bytes);
uint64_t or_sweep_index(or_handle* h);
int   or_set_sweep_index(or_handle* h, uint64_t s);
/* rho_i(tau_k) = eta g_sigma(I eta) of the interval that holds slice
   tau_k = k beta / K on site i (Supplement S-I); out[i*K + k]. */
int   or_rho_slices(or_handle* h, int32_t K, double* out);
/* Supplement S-I, resolved by the component of Q (a = 0: Q_b = b, a = 1:
   Q_b+ = b+) at the K slices tau_k = k beta / K:
   out[(s K + k) 2 + a] = rho_a; iv[s K + k] = event index of the lower
   vertex leg of the slice's interval, -1 on a site without legs (two slices
   of one site share an interval iff their iv are equal).                  */
int   or_rho_alpha(or_handle* h, int32_t K, double* out, int32_t* iv);
/* two-point densities of one site: out[((s K + k1) K + k2) 4 + a1 2 + a2]
   for Q_a1 at slice k1 and Q_a2 at slice k2 (0 when k1 == k2).           */
int   or_rho_pair(or_handle* h, int32_t K, double* out);

/* Supplement S-I n-point functions resolved by the component of Q at
   arbitrary times (several points may share an interval): tuple j holds n
   points (site, slice k in 0..K-1, component a: 0 = b, 1 = b+) at
   pts[(j n + c) 3 + 0..2]; out[j] = <Q_a1(X_1) ... Q_an(X_n)> estimated as
   eta^-n times the product over the intervals holding the points of their
   joint density, averaged over the K cyclic shifts of all slices.        */
int   or_npoint_alpha(or_handle* h, int32_t K, int32_t n, int64_t m, const int32_t* pts, double* out);
/* joint density of g operators Q_a[0..g) on one interval with end states p
   (below) and q (above) and M worm points, point j having M1[j] worm points
   below it (increasing); p < 0: a site without legs, M1[j] = time point pk */
double or_interval_density(int p, int q, uint64_t M, int g, const uint64_t* M1, const int* a, double eta, double XW);

/* building blocks, exported for the pins */
void  or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_exp_det(double x);
double or_expm1_det(double x);
/* ziggurat tables: X[257], F[257], W[256], K[256], R, v */
void  or_zig_tables(double* X, double* F, double* W, uint64_t* K, double* R, double* v);
/* n exponential deviates from the stream (key, unit, c2, sweep) */
int   or_exp_deviates(uint64_t seed, uint32_t unit, uint32_t c2, uint32_t sweep,
                      int64_t n, double* out);
/* worm-number sampler (Eq. 1): M worm grid points, parity sigma, inverse
   scale SW = 2^59/(beta eta); writes sorted offsets, returns count or -1. */
int   or_sample_worms(uint64_t seed, uint32_t unit, uint32_t c2, uint32_t sweep,
                      uint64_t M, int sigma, double SW, uint64_t* offs, int max);
/* Step 1's law (Eq. 3): P(s') of the new boundary state for end states p
   (below) and q (above), M1 worm grid points above the boundary and M2 below,
   x = M XW; out[s'] for s' = 0, 1 */
void  or_pdom(int p, int q, uint64_t M1, uint64_t M2, double XW, double out[2]);
/* derived per-instance tables (for comparison with the product's own) */
int   or_tables(const or_params* p, double* d4, double* Dmax, uint64_t* TV4,
                uint64_t* TH256, double* SV, double* SW);

#ifdef __cplusplus
}
#endif
#endif
