/*
 * pmwa.h -- C ABI of libpmwa.so: the parallelized multiple-worm algorithm
 * (PMWA) Monte Carlo sweep for the hard-core Bose-Hubbard model on one GB300.
 *
 * Method: Masaki-Kato, Suzuki, Harada, Todo, Kawashima, "Parallelized Quantum
 * Monte Carlo Algorithm with Nonlocal Worm Updates" (arXiv:1307.0328).
 * The simulated Hamiltonian is H_eta = H - eta Q with Q = sum_i (b_i + b_i^+)
 * (introduction; Eq. 5 for H, read as -t sum_<ij>(b+_i b_j + h.c.)
 * + V sum_<ij> n_i n_j - mu sum_i n_i and written per bond with
 * -(mu/4)(n_i + n_j)).  One MC step ("sweep") is the paper's pseudo code:
 *   Step 2  spatial-boundary update of the vertices on bonds between domains
 *           (Eq. 4), every `exchange_every` sweeps, followed there by Step 3
 *           on those bonds;
 *   Step 3  vertex phase on all other bonds;
 *   Step 4  worm creation on every interval (Eq. 1);
 *   Step 5  N_cycle passes of worm scattering (Eq. 2);
 *   Step 6  measurement (energy, density, order parameter <Q>, and the
 *           worm-density estimator of Supplement S-I).
 * All domains live in one GPU's HBM; the paper's neighbour messages become
 * kernels that read the neighbour's sites directly.
 *
 * Conventions for every call:
 *   - Status: 0 = PMWA_OK, else one of the PMWA_E* codes; pmwa_strerror()
 *     names them.  Calls never abort the process.
 *   - Memory: the caller owns the params, the device arena and every output
 *     buffer.  The handle holds small host tables only.
 *   - Streams: work is queued on the stream given to pmwa_create (a
 *     cudaStream_t passed as void*; NULL = legacy default stream).  Calls that
 *     return data to the host are synchronous; pmwa_sweep is synchronous too
 *     (it reports device-side errors).
 *   - Layout of the configuration (canonical export format, identical to the
 *     CPU oracle's): u64 n_sites, then for every site i = x + Lx*y a u64
 *     header (count | base_state << 63) followed by `count` u64 event keys
 *     sorted in time.  Key bits 63..5: time-grid index m (2^59 points per
 *     beta); bits 4..2: tag (0..5 vertex leg of the bond of class tag, 7
 *     worm); bit 1: state below (vertex leg) or direction up (worm); bit 0:
 *     state above.
 */
#ifndef PMWA_H
#define PMWA_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PMWA_OK          0
#define PMWA_EINVAL      1  /* bad parameter or buffer size                       */
#define PMWA_ECAPACITY   2  /* a fixed-capacity list would overflow               */
#define PMWA_ETIMEOUT    3  /* a bounded device loop reached its cap              */
#define PMWA_ECUDA       4  /* a CUDA runtime call failed                         */
#define PMWA_EINVARIANT  5  /* the configuration breaks an invariant              */
#define PMWA_EROWS       6  /* measurement row buffer full: call pmwa_measure     */

/* When a kernel reports PMWA_ECAPACITY, PMWA_ETIMEOUT or PMWA_EINVARIANT, it
   has stopped part-way and the handle's configuration is undefined: the
   kernels queued after it on that instance leave at once, and pmwa_sweep,
   pmwa_tile, pmwa_boundary, pmwa_rho_slices*, pmwa_green, pmwa_export*, pmwa_check and
   pmwa_batch_sweep (for an active instance) return PMWA_EINVARIANT until
   pmwa_import restores a configuration.  Every per-site event count stays
   within the site's slot at all times, so no call reads out of bounds. */

/* Simulation parameters (problem statement: introduction, Eq. 5; domains:
   Supplement S-II; Step-5 passes: Step 6 of the pseudo code). */
typedef struct {
  int32_t  Lx, Ly;          /* periodic square lattice, both >= 2                 */
  double   beta, t, V, mu, eta; /* beta > 0, t >= 0, eta > 0                      */
  uint64_t seed;            /* Philox4x32-10 key of every random draw             */
  int32_t  dom_x, dom_y;    /* sites per domain; 0 = whole axis; must divide L;
                               >= 2 when an axis has several domains              */
  int32_t  exchange_every;  /* K >= 1: Step 2 runs when sweep % K == 0            */
  int32_t  n_cycle;         /* Step-5 passes per sweep, 0..4095                   */
  int32_t  sub_block;       /* Step-5 shifted sub-block edge B (even); 0 = domain */
  int32_t  init;            /* 0: empty lattice; 1: floor(N/2) particles placed by
                               a Fisher-Yates permutation of stream init_seed;
                               2: checkerboard, sites with x + y even occupied    */
  uint64_t init_seed;
  double   c_off;           /* diagonal vertex weight offset; < 0 means t/2       */
  uint32_t replica;         /* 0..65535, mixed into every Philox counter          */
  int32_t  cap_site;        /* events per site slot; 0 = sized from beta, t, V, mu */
  int32_t  rows_cap;        /* measurement rows held on the device; 0 = 4096      */
  int32_t  legs_hint;       /* mean vertex legs per site, e.g. 2 n_v / N from a
                               pilot run: sizes the shared-memory leg table of a
                               domain tighter than the bound 4 beta (D + t), which
                               leaves room to stage the domain's configuration in
                               shared memory; 0 = the bound.  Too small a hint
                               makes a sweep return PMWA_ECAPACITY.            */
  int32_t  dom_tau;         /* temporal domains N_beta (Supplement S-II), 0..64;
                               0 and 1 mean one domain spanning beta.  With
                               N_beta > 1, boundary k sits at the grid point
                               floor(k 2^59 / N_beta) of every site; Step 1
                               (Eq. 3) runs when sweep % K == 0, before Step 2 */
  int32_t  reserved[1];     /* must be 0                                          */
  double   vertex_window;   /* on-the-fly vertex generation (the paper's closing
                               discussion of extensions): 0 = the vertex phase
                               everywhere; w in (0, 1] = the vertex phase of a
                               bond only at grid points within w beta of a worm
                               of the current configuration on either of its
                               sites (diagonal vertices elsewhere stay).  The
                               windows depend on the worms alone, which Step 3
                               does not move, so the distribution is kept.  Not
                               in replica batches.                               */
} pmwa_params;

/* One row per sweep (Step 6 measurement after Step 5). */
typedef struct {
  uint64_t sweep;   /* sweep index                                              */
  uint64_t n_v;     /* vertices (diagonal + kinks) on all bonds                 */
  uint64_t n_k;     /* kinks                                                    */
  uint64_t n_w;     /* worms                                                    */
  uint64_t occ_lo;  /* sum over sites of occupied imaginary time, in units of   */
  uint64_t occ_hi;  /*   beta / 2^62, as a 128-bit integer (hi:lo)              */
  double   q_impr;  /* Supplement S-I: sum over intervals of x g_sigma(x),
                       x = I eta, g_0 = tanh, g_1 = coth; <Q> = q_impr/(beta eta) */
  uint32_t w_dom_min; /* fewest worms held by one (space-time) domain after Step 5 (the
                         paper's health figure of O(10)-O(100) worms per domain,
                         discussion of Fig. 3)                                  */
  uint32_t dom_empty; /* domains without a worm after Step 5                   */
} pmwa_row;

typedef struct pmwa_handle pmwa_handle;

/* Bytes of device arena that pmwa_create needs for these parameters
   (0 if the parameters are invalid). */
size_t pmwa_footprint(const pmwa_params* p);

/* Validate p, carve the caller's device arena (arena_bytes >=
   pmwa_footprint(p), 256-byte aligned), build the host tables (directed-loop
   thresholds of Eq. 2, vertex thinning thresholds, ziggurat), write the
   initial configuration, and return a handle.  The arena must stay valid
   until pmwa_destroy.  stream: cudaStream_t or NULL. */
int pmwa_create(const pmwa_params* p, void* dev_arena, size_t arena_bytes,
                void* stream, pmwa_handle** out);

/* Run n_sweeps MC steps (pseudo code Steps 1-6; Step 1 only with temporal
   domains, dom_tau > 1).  One measurement row per sweep.
   PMWA_EROWS if the rows would not fit: drain them with pmwa_measure first.
   With temporal domains the worms of Step 5 turn round at the temporal
   boundaries and every leg of Eq. 2 ends there; Step 4 draws the worms of
   the intervals delimited by the vertex legs and the boundaries; Step 2's
   legs end there too; and the Step-5 schedule runs each sub-block of each
   temporal slab as its own chain (Philox unit = sub-block id * N_beta +
   slab).  The Step-6 estimator q_impr sums over those intervals; the slice
   estimators (pmwa_rho_*, pmwa_green*, pmwa_npoint*) use the intervals
   between vertex legs; both are unbiased. */
int pmwa_sweep(pmwa_handle* h, int64_t n_sweeps);

/* Fine-grained steps, for parity checks: Step 1 (temporal boundaries,
   Eq. 3; nothing with one temporal domain) and Step 2 (+ Step 3 on the
   boundary bonds) regardless of the sweep index; and Steps 3..stop_after of
   one sweep (stop_after in 3..6; 6 also records a row).  None advances the
   sweep index.  Step 1: every boundary k of a site, in order k = 0, 1, ...,
   takes the new state s' with probability f_{q s'}(I1) f_{s' p}(I2) /
   f_{q p}(I) (I2 from the nearest vertex leg or boundary below, state p above
   it; I1 up to the nearest one above, state q below it; worms ignored), and
   the worms of I2 and I1 are drawn anew (Eq. 1); one warp per site. */
int pmwa_temporal(pmwa_handle* h);
int pmwa_boundary(pmwa_handle* h);
int pmwa_tile(pmwa_handle* h, int32_t stop_after);

/* Copy up to max_rows pending rows to host memory `rows` (caller-owned,
   max_rows rows), oldest first, and drop them from the device buffer;
   *n_rows = number copied.  The freed rows are cleared on the handle's
   stream before the call returns (later sweeps add into them), so the call
   is ordered with sweeps on any stream.  Synchronous. */
int pmwa_measure(pmwa_handle* h, pmwa_row* rows, int64_t max_rows, int64_t* n_rows);

/* Supplement S-I worm density at K equal-time slices tau_k = k beta / K:
   host_out[i*K + k] = eta g_sigma(I eta) of the interval (between vertex
   legs) that holds tau_k on site i.  host_out holds N*K doubles. */
int pmwa_rho_slices(pmwa_handle* h, int32_t K, double* host_out);

/* Equal-time Green functions of Q from the worm densities (Supplement S-I:
   <prod_k Q(X_k)> = eta^-n <prod_k rho(X_k)> when no two X_k share an
   interval, which holds for distinct sites at equal time), averaged over
   sites and the K slices tau_k = k beta / K of the current configuration:
   gx[r-1] = <Q_i Q_{i+r x}>, gy[r-1] = <Q_i Q_{i+r y}> for r = 1..rmax
   (rmax <= min(Lx, Ly)/2), and *plaq = <Q_i Q_{i+x} Q_{i+y} Q_{i+x+y}>, the
   4-point function on a plaquette.  Host outputs; uses the arena's idle
   next-configuration slots as scratch. */
int pmwa_green(pmwa_handle* h, int32_t K, int32_t rmax, double* gx, double* gy, double* plaq);

/* The same values as pmwa_rho_slices, for callers that cannot allocate
   device memory while they run (for example a serving loop whose memory is
   owned by another allocator, or one that has promised its pool no new
   blocks): the device scratch of this call is a fixed array inside the
   library, not the caller's arena, and nothing is allocated or freed.  The
   paper has no counterpart.  Limit: N*K <= 2^20 doubles (8 MiB, held on every
   GPU that loads the library until exit); larger requests return
   PMWA_EINVAL.  The handle's device must be current.  The first call on a
   device looks up the array's device address and keeps it for the process;
   make that first call before any stream capture.  The kept address belongs
   to the device's primary context: after cudaDeviceReset (or anything else
   that destroys that context) it is stale, and the handles created before
   are unusable anyway, so do not call this entry point again in that
   process.  Calls that overlap on the GPU share the array and race; each
   call overwrites every value it returns. */
int pmwa_rho_slices_static(pmwa_handle* h, int32_t K, double* host_out);

/* Supplement S-I n-point functions of listed site tuples at equal time:
     host_out[j] = < Q_i1(tau) ... Q_in(tau) > = eta^-n < rho_i1(tau) ... rho_in(tau) >,
   averaged over the K slices tau_k = k beta / K, for tuple j of n sites
   host_sites[j n + c] (row-major, m tuples, caller-owned), rho the density
   of pmwa_rho_slices.  Distinct sites never share an interval, so the
   densities multiply; a tuple that names one site twice, or a site outside
   0..N-1, returns PMWA_EINVAL.  1 <= n <= 16, m >= 0; host_out holds m
   doubles (caller-owned).  Per tuple: for each slice the product over the
   sites in tuple order, summed over the slices in order, divided by K and
   then by eta^n.  Scratch: the idle next-configuration slots (the densities,
   8 K bytes per site, then chunks of tuples); PMWA_EINVAL when the densities
   leave no room for one tuple.  Synchronous. */
int pmwa_npoint(pmwa_handle* h, int32_t K, int32_t n, int64_t m, const int32_t* host_sites, double* host_out);

/* Supplement S-I resolved by the component of Q = b + b+ (a = 0: Q_b = b,
   which takes a site from 1 to 0; a = 1: Q_b+ = b+): at the K slices
   tau_k = k beta / K of every site,
     rho_a(X) = eta <q| e^{I2 eta Q} Q_a e^{I1 eta Q} |p> / <q| e^{I eta Q} |p>,
   where the slice X splits the interval I between the vertex legs around it
   (p the state above the lower leg, q the state below the upper one) into
   I1 below X and I2 above; rho_b + rho_b+ is the value of pmwa_rho_slices.
   A site without vertex legs gets the trace form eta tanh(beta eta) / 2 for
   both components.  host_rho[(s K + k) 2 + a] (N K 2 doubles, caller-owned);
   host_iv[s K + k] (N K int32, caller-owned, may be NULL) = index of the
   interval's lower leg in the site's time-ordered events, -1 on a site
   without legs: two slices of one site lie on the same interval iff their
   iv are equal, and then their joint density is not the product of the two
   (pmwa_green_tau handles that case).  Products of densities at points on
   different intervals estimate eta^n <prod Q_a(X)> (Supplement S-I).
   Scratch: the idle next-configuration slots (8 cap bytes per site), filled
   by chunks of sites.  Synchronous. */
int pmwa_rho_alpha(pmwa_handle* h, int32_t K, double* host_rho, int32_t* host_iv);

/* Unequal-time single-particle Green function of H_eta from the densities
   above (Supplement S-I):
     host_g[(d (rmax + 1) + r) K + dk] = G_d(r, dk)
       = < b_{i + r e_d}(tau_k + dk beta / K) b+_i(tau_k) >,
   averaged over sites i and slices k, d = 0 (x) or 1 (y), r = 0..rmax,
   dk = 0..K-1 (tau cyclic in beta).  Points on different intervals take the
   product of their densities / eta^2; two points on one interval of a site
   (r = 0; the case the paper leaves to later work) take both operators inside
   the interval's matrix element,
     eta^2 <q| e^{Ic Q} Q_U e^{Ib Q} Q_L e^{Ia Q} |p> / <q| e^{I Q} |p> / eta^2
   (L the lower point going up from the lower leg, Ia, Ib, Ic the parts of I
   from the bottom), and on a site without legs the cyclic trace form.  G at
   r = dk = 0 (both operators at one point) is not estimated and is 0; the
   r = 0 row is the same for d = 0 and 1.  1 <= K <= 64,
   0 <= rmax <= min(Lx, Ly) / 2; host_g holds 2 (rmax + 1) K doubles
   (caller-owned).  Scratch: the idle next-configuration slots hold every
   site's densities when rmax >= 1, so PMWA_EINVAL unless 16 K bytes per
   site plus the sums fit in 8 cap bytes per site (K <= cap / 2 about; cap
   from pmwa_slot_capacity).  Synchronous. */
int pmwa_green_tau(pmwa_handle* h, int32_t K, int32_t rmax, double* host_g);

/* Supplement S-I n-point functions resolved by the component of Q at
   arbitrary times, for listed tuples of points: tuple j holds n points
   (site s, slice k in 0..K-1, component a: 0 = b, 1 = b+) at
   host_pts[(j n + c) 3 + 0..2] (row-major, m tuples, caller-owned), and
     host_out[j] = < T Q_a1(X_1) ... Q_an(X_n) >
                 = eta^-n < prod over intervals of the joint density of the
                   points on that interval >,
   averaged over the K cyclic shifts of all slices (X_c at tau = ((k_c + t)
   mod K) beta / K, t = 0..K-1; the thermal state is invariant under the
   shift).  Points on different intervals multiply their densities (the
   densities of pmwa_rho_alpha); several points on one interval take all
   their operators inside the interval's matrix element,
     eta^g <q| e^{I_g Q} Q_a[g-1] ... e^{I_1 Q} Q_a[0] e^{I_0 Q} |p> / <q| e^{I Q} |p>,
   in time order going up from the lower leg (the case the paper leaves to
   later work; the same derivation as the single point with g delta
   functions), and on a site without legs the cyclic trace.  The product
   over the groups runs in order of first appearance, the sum over shifts in
   order, then / K / eta^n.  PMWA_EINVAL for a site or slice out of range, a
   component other than 0 or 1, or one (site, slice) named twice in a tuple;
   1 <= n <= 16, 1 <= K <= 2^20.  Scratch: the idle next-configuration slots
   (12 n + 8 bytes a tuple, in chunks).  Synchronous. */
int pmwa_npoint_alpha(pmwa_handle* h, int32_t K, int32_t n, int64_t m, const int32_t* host_pts, double* host_out);

/* Canonical configuration (format in the header comment) to / from host
   memory.  pmwa_export_bytes gives the size; pmwa_import checks the
   invariants and the per-site capacity. */
int pmwa_export_bytes(pmwa_handle* h, size_t* bytes);
int pmwa_export(pmwa_handle* h, void* host_buf, size_t bytes);
int pmwa_import(pmwa_handle* h, const void* host_buf, size_t bytes);

/* Invariants of the current configuration, checked on the device (one warp
   per site; the worldline representation of the paper's introduction and
   Steps 3-5 keep them all):
     PMWA_CHECK_CAPACITY      a site's count exceeds its slot;
     PMWA_CHECK_TAG           a key is neither a bond leg (tags 0..5) nor a worm (7);
     PMWA_CHECK_ORDER         a site's times do not strictly increase;
     PMWA_CHECK_CONTINUITY    the state above an event differs from the state
                              below the next one (cyclic in time);
     PMWA_CHECK_BASE          the base state differs from the state above the last event;
     PMWA_CHECK_BOND          a leg's tag names no bond of its site;
     PMWA_CHECK_PARTNER       the bond's other site has no leg at the same time;
     PMWA_CHECK_CONSERVATION  a vertex does not conserve particles (s0 + s1 != s2 + s3).
   Returns PMWA_OK with *site = -1, *what = 0 when all hold; PMWA_EINVARIANT
   with the lowest failing site and the lowest failing code at that site; on
   a handle whose configuration is undefined (see above) PMWA_EINVARIANT with
   *site = -1.  pmwa_import checks the first five and the capacity on the
   host; this call checks all eight on the device, for example after every
   step of a debugging run.  Reads stay inside the slots whatever the
   configuration.  Synchronous; uses the idle next-configuration slots as
   scratch.  Cost: one pass over the configuration. */
#define PMWA_CHECK_CAPACITY     1
#define PMWA_CHECK_TAG          2
#define PMWA_CHECK_ORDER        3
#define PMWA_CHECK_CONTINUITY   4
#define PMWA_CHECK_BASE         5
#define PMWA_CHECK_BOND         6
#define PMWA_CHECK_PARTNER      7
#define PMWA_CHECK_CONSERVATION 8
int pmwa_check(pmwa_handle* h, int64_t* site, int32_t* what);

/* Sweep index (the Philox counter word of every draw of a sweep). */
int pmwa_get_sweep(pmwa_handle* h, uint64_t* sweep);
int pmwa_set_sweep(pmwa_handle* h, uint64_t sweep);

/* Release the handle (the arena stays the caller's). */
int pmwa_destroy(pmwa_handle* h);

/* Change N_cycle (Step 6 of the pseudo code: Step 5 is repeated N_cycle
   times) of an instance, 0..4095. */
int pmwa_set_n_cycle(pmwa_handle* h, int32_t n_cycle);

/* ---- batches: many independent instances, one launch per kernel per sweep.
   Each instance keeps exactly the configuration it would have alone: every
   random draw is keyed by its own seed, replica id, sweep and unit, so a
   batched sweep and n plain sweeps give identical bytes.  No paper
   counterpart (the paper runs one instance on many processors); this is the
   replica-batching pattern.  p points to n parameter sets; the arena holds
   the batch tables and every instance's own arena. */
typedef struct pmwa_batch pmwa_batch;
size_t pmwa_batch_footprint(const pmwa_params* p, int32_t n);
int pmwa_batch_create(const pmwa_params* p, int32_t n, void* dev_arena, size_t arena_bytes,
                      void* stream, pmwa_batch** out);
/* n_sweeps MC steps of every active instance (one measurement row each). */
int pmwa_batch_sweep(pmwa_batch* b, int64_t n_sweeps);
/* Capture `sweeps` batched sweeps in a CUDA graph (0 = no graph); later
   pmwa_batch_sweep calls whose count is a multiple of it replay the graph. */
int pmwa_batch_graph(pmwa_batch* b, int32_t sweeps);
/* The instance's handle (for pmwa_measure, pmwa_export, pmwa_import, ...;
   pmwa_sweep on it advances that instance alone: the plain path). */
int pmwa_batch_instance(pmwa_batch* b, int32_t i, pmwa_handle** h);
/* An inactive instance is skipped by pmwa_batch_sweep. */
int pmwa_batch_set_active(pmwa_batch* b, int32_t i, int32_t on);
int pmwa_batch_set_n_cycle(pmwa_batch* b, int32_t i, int32_t n_cycle);
/* Device time (CUDA events on the stream) of the last pmwa_batch_sweep. */
int pmwa_batch_last_ms(pmwa_batch* b, double* ms);
int pmwa_batch_destroy(pmwa_batch* b);
/* A batch over existing handles (each created by pmwa_create in its own
   arena): the configurations stay where they are, so the set of instances
   advanced together can change between calls without moving any state (the
   serving pattern).  The arena holds only the batch tables,
   pmwa_batch_tables_bytes(hs, n) bytes.  Destroying such a batch leaves the
   handles to the caller. */
size_t pmwa_batch_tables_bytes(pmwa_handle* const* hs, int32_t n);
int pmwa_batch_from_handles(pmwa_handle* const* hs, int32_t n, void* dev_arena, size_t arena_bytes,
                            void* stream, pmwa_batch** out);

/* Host tables derived from p, for comparison with an independent
   implementation: d4[4] diagonal vertex weights d(s) = C - E(s); *D = max d;
   tv4[4] thinning thresholds floor(d/D 2^32); th256[16*4*4] directed-loop
   cumulative exit thresholds (Eq. 2) by root state S, entry leg i, exit leg
   j; *sv = 2^59/(beta D); *sw = 2^59/(beta eta); zig: X[257], F[257],
   W[256] doubles and K[256] u64 of the exponential ziggurat (any may be NULL). */
int pmwa_tables(const pmwa_params* p, double* d4, double* D, uint64_t* tv4,
                uint64_t* th256, double* sv, double* sw,
                double* zig_x, double* zig_f, double* zig_w, uint64_t* zig_k);

/* The shared-memory plan of a domain for these parameters: *smem bytes per
   CTA, *legcap vertex legs in its leg table, *oldcap events of the current
   configuration staged in shared memory for Steps 3 (0: read from HBM).
   Host only; returns PMWA_EINVAL for invalid parameters or a domain that
   does not fit.  Any pointer may be NULL. */
int pmwa_tile_plan(const pmwa_params* p, int32_t* smem, int32_t* legcap, int32_t* oldcap);

/* Events each site's slot holds (the configuration's per-site capacity,
   fixed at create from the parameters).  PMWA_EINVAL for invalid
   parameters. */
int pmwa_slot_capacity(const pmwa_params* p, int32_t* cap);

/* Shared memory (bytes) the sweep kernel needs per domain for these
   parameters, 0 if a domain does not fit on one SM (a domain-shape tuner
   uses it).  Host only. */
int32_t pmwa_tile_smem(const pmwa_params* p);

/* Per-kernel timing with CUDA events recorded on the handle's stream around
   every launch (enable = 1 turns it on, 0 off and clears).  pmwa_profile_read
   synchronises and returns, for kernel k = 0 spatial boundary (Step 2),
   1 sweep kernel (Steps 3-6), 2 temporal boundaries (Step 1), 5 rho slices,
   and 6 the device span of each whole sweep of pmwa_sweep, the summed device
   milliseconds ms[k] and the number of launches[k] since the last read
   (n >= 7 entries each; 3 and 4 are unused), then clears them.  No paper
   counterpart: measurement plumbing. */
int pmwa_profile(pmwa_handle* h, int32_t enable);
int pmwa_profile_read(pmwa_handle* h, double* ms, int64_t* launches, int32_t n);
/* SM clock cycles spent by the sweep kernel in each of its phases, summed
   over its CTAs since the last call while profiling is on: 0 vertex
   candidates (Step 3), 1 leg merge (Step 3), 2 worm creation (Step 4),
   3 scattering (Step 5) outside the block-wide passes (all of it for a
   domain of at most 32 worms, whose passes run in one warp), 4 output +
   measurement (Step 6), 5 per-pass set-up of the block-wide passes
   (grouping, move descriptors, random words), 6 their moves; 7 (a count,
   not cycles) the rounds of independent moves the block-wide passes took;
   n >= 8 entries,
   cleared after reading.  No paper counterpart: measurement plumbing. */
int pmwa_profile_phases(pmwa_handle* h, uint64_t* cycles, int32_t n);

/* ---- Step 6: observables from the measurement rows (host only).
   Definitions (pseudo code Step 6; Supplement S-I; model of Eq. 5 written per
   bond as E(n_a, n_b) = V n_a n_b - (mu/4)(n_a + n_b), C = max E + c_off,
   N sites, N_b = 2 N bonds):
     E      = (N_b C - n_v / beta) / N            energy of H per site
     E_eta  = E - eta Q_impr                       energy of H_eta = H - eta Q per site
     n      = occupied time / (beta N)             density
     Q_raw  = n_w / (beta eta N)                   <Q>/N from the worm count
     Q_impr = q_impr / (beta eta N)                <Q>/N, Supplement S-I estimator
     kin    = n_k / (beta t N_b)                   <b+_i b_j + h.c.> per bond (0 if t = 0)
   pmwa_row_observables writes these six per row, out[r * PMWA_SERIES + k]
   with k = PMWA_S_E, ... (n_rows * PMWA_SERIES doubles, caller-owned). */
#define PMWA_SERIES   6
#define PMWA_S_E      0
#define PMWA_S_E_ETA  1
#define PMWA_S_N      2
#define PMWA_S_Q_RAW  3
#define PMWA_S_Q_IMPR 4
#define PMWA_S_KIN    5
int pmwa_row_observables(const pmwa_params* p, const pmwa_row* rows, int64_t n_rows, double* out);

/* Means and binned standard errors of the six series over the first
   bins * floor(n_rows / bins) rows (the remainder at the end is left out):
   the rows are cut into `bins` consecutive bins of equal length, x_err =
   sqrt(sum_b (m_b - m)^2 / (bins (bins - 1))) over the bin means m_b.
   Also the mean vertices and worms per sweep and the worms-per-domain figures
   the paper uses to judge a decomposition (O(10)-O(100) worms per domain and a
   small chance of an empty domain; discussion of Fig. 3): the mean over the
   used rows of n_w / domains, the smallest w_dom_min, and the fraction of
   (domain, sweep) pairs without a worm.  Domains = (Lx / dom_x)(Ly / dom_y)
   times the temporal domains.
   2 <= bins <= n_rows; PMWA_EINVAL otherwise or for invalid parameters. */
typedef struct {
  int64_t rows;                 /* rows used                                   */
  int32_t bins, pad;
  double  E, E_err;
  double  E_eta, E_eta_err;
  double  n, n_err;
  double  Q_raw, Q_raw_err;
  double  Q_impr, Q_impr_err;
  double  kin, kin_err;
  double  n_v, n_w;             /* mean vertices and worms per sweep            */
  double  w_dom_mean;           /* mean worms per domain                        */
  double  w_dom_min;            /* fewest worms seen in one domain              */
  double  dom_empty_frac;       /* fraction of (domain, sweep) pairs without worms */
} pmwa_obs;
int pmwa_observables(const pmwa_params* p, const pmwa_row* rows, int64_t n_rows, int32_t bins, pmwa_obs* out);

/* N_cycle, the Step-5 passes per sweep, by the rule that every part of the
   space-time is visited about once per sweep (pseudo code Step 5): a move
   lands a worm on one vertex leg, a sweep holds 2 n_v legs and n_w worms move
   per pass, so N_cycle = ceil(2 <n_v> / <n_w>) with the means over the given
   rows (e.g. the second half of a pilot), <n_w> at least 1; with no rows
   (n_rows = 0) the a-priori estimate from <n_v> = N_b beta (d_mean + t/2)
   (d_mean the mean of d(s) = C - E(s) over the four states) and
   <n_w> = beta eta N / 2.  Capped to 1..512.  Host only. */
int pmwa_n_cycle(const pmwa_params* p, const pmwa_row* rows, int64_t n_rows, int32_t* n_cycle);

/* Caps of the bounded device loops of this handle: words drawn for one
   exponential deviate (1..64, the specification's 64 by default) and
   proposals of the Eq. 1 worm-number sampler (1..128, default 128).  The
   defaults are part of the deterministic specification; smaller caps exist
   to exercise the PMWA_ETIMEOUT path, which then leaves the configuration
   undefined until pmwa_import (see above).  Takes effect at the next plain
   call on the handle (a batch copies its instances' settings when it is
   created).  No paper counterpart: test plumbing. */
int pmwa_set_loop_caps(pmwa_handle* h, int32_t zig_words, int32_t worm_tries);

/* n Philox4x32-10 blocks computed by the device code every kernel draws
   from: host_in[6 j .. 6 j + 6) = counter words c0..c3 and key words k0, k1
   of block j, host_out[4 j .. 4 j + 4) = its four output words
   (caller-owned host buffers).  Scratch: the handle's idle
   next-configuration slots (40 bytes per block; PMWA_EINVAL beyond them).
   Synchronous.  No paper counterpart: it lets a test compare the device
   generator with published known-answer vectors. */
int pmwa_philox_blocks(pmwa_handle* h, int64_t n, const uint32_t* host_in, uint32_t* host_out);

const char* pmwa_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif
