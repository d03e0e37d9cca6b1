// pmwa_internal.h -- state shared by the host side (pmwa_host.cpp) and the
// CUDA kernels (pmwa_kernels.cu) of libpmwa.so.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/pmwa.h"

namespace pmwa {

constexpr uint64_t kTwo59 = uint64_t(1) << 59;
constexpr uint64_t kTwo62 = uint64_t(1) << 62;
constexpr uint64_t kTwo32 = uint64_t(1) << 32;

// Philox counter word c2 = phase | pass << 4 | replica << 16.
enum Phase : uint32_t { kInit = 1, kBx = 2, kBy = 3, kVertex = 4, kRegen = 5, kScatter = 6, kTemporal = 7 };

// Error word layout on the device: first error code wins (atomicCAS).
struct DevErr {
  int code;
  int where;
};

// A mean grid spacing S of a Bernoulli process (Steps 3 and 4) in the form
// the integer gap arithmetic uses: S = m 2^(sh - 122), m in [2^63, 2^64) the
// binary64 mantissa of S at the top of a u64, sh = 121 - floor(log2 S), so
// that E S = (E 2^58) m / 2^sh for a fixed-point deviate E 2^58.
struct GridScale {
  uint64_t m;
  int sh;
};

// Everything a kernel needs, passed by value.
struct Dev {
  // geometry
  int Lx, Ly, N, dom_x, dom_y, ndx, ndy, ndom;
  int sub_block, n_cycle;
  int cap;      // events per site slot
  int capb;     // candidate vertices per bond (Step 3)
  int wcap;     // worms per domain in the shared-memory worm table
  int legcap;   // vertex legs per domain in shared memory
  int poolcap;  // Step-3 candidates per domain in shared memory
  // shared-memory carve-up of the tile kernel (byte offsets)
  int sm_th, sm_zig, sm_off, sm_base, sm_bcnt, sm_boff, sm_misc, sm_nbr, sm_sub, sm_tinfo, sm_leg, sm_wcnt, sm_pool,
      sm_worm, sm_idx, sm_ord, sm_wsb, sm_wrk, sm_rw, sm_bkt, sm_cnt, sm_fill, sm_total;
  int sm_soff, sm_old;  // staged current configuration of the domain (phases 1-2)
  int sm_part;          // [legcap] u16: index of each vertex leg's partner leg (Step 5)
  int use_part;         // 1: the partner table is planned; 0: Step 5 searches for partners
  int oldcap;           // events it can hold; 0 = read the configuration from HBM
  unsigned long long* phase_cycles;  // 8 counters when profiling, else null
  // random numbers
  uint32_t key0, key1, replica, sweep;
  // model
  double beta, eta, SV, SW, XW;
  GridScale SVs, SWs;  // SV and SW in the fixed-point form of the grid gaps
  GridScale XQ;        // beta eta 2^5: x 2^64 = (I m) >> sh for an interval of I worm points
  uint64_t SWI;
  int has_vertices;
  uint64_t TV[4];
  double dvw[4];    // diagonal vertex weights d(s), s = na | nb << 1
  double tkink;     // kink weight t
  float dvwf[4], tkinkf, XWf;  // the same rounded to binary32 (heat-bath pre-decision)
  // buffers
  uint64_t* keyA;   // current configuration: N slots of cap keys
  uint32_t* cntA;   // count | base << 31
  uint64_t* keyB;   // next configuration
  uint32_t* cntB;
  const uint64_t* TH;  // 16*4*4 directed-loop thresholds
  DevErr* err;
  pmwa_row* rows;
  int row;
  // both configuration buffers (keyA/keyB above are the current selection)
  uint64_t* bufk[2];
  uint32_t* bufc[2];
  int exchange_every;
  // caps of the bounded device loops (a stuck loop ends in PMWA_ETIMEOUT):
  // words of one exponential deviate (ziggurat) and proposals of the Eq. 1
  // sampler; the deterministic specification fixes 64 and 128, smaller
  // values exist only to exercise the error path
  int zig_cap, worm_tries;
  // temporal domains N_beta (1: none); boundary k at grid point
  // m_k = k tq + (k tr) / ntau with 2^59 = tq ntau + tr, i.e. floor(k 2^59 / ntau)
  int ntau;
  uint64_t tq, tr;
  // on-the-fly vertex generation: the vertex phase of a bond only within
  // win_half worm grid points of a worm on its sites (0: everywhere)
  uint64_t win_half;
  int sm_wmo, sm_wm;  // shared-memory offsets of the windows' worm index (k_tile)
};

// Per-instance state at the start of a batched call: the sweep index, the
// next free measurement row, which buffer holds the current configuration,
// and whether the instance takes part.
struct BatchBase {
  uint32_t sweep0;
  int row0;
  int flip;
  int active;
};

// An instance's parameters advanced to sweep iteration `it` of a batched call
__host__ __device__ inline Dev at_iteration(const Dev& d0, const BatchBase& b, int it) {
  Dev d = d0;
  const int cur = (b.flip + it) & 1;
  d.keyA = d0.bufk[cur];
  d.cntA = d0.bufc[cur];
  d.keyB = d0.bufk[cur ^ 1];
  d.cntB = d0.bufc[cur ^ 1];
  d.sweep = b.sweep0 + uint32_t(it);
  d.row = b.row0 + it;
  return d;
}


// Exponential ziggurat tables, built on the host (pmwa_host.cpp).
struct Zig {
  double X[257], F[257], W[256];
  double S[256];     // slope (F[i] - F[i+1]) / (X[i] - X[i+1]) of strip i's chord (i >= 1)
  uint64_t K[256];
  uint64_t XF[256];  // X[i] 2^58 (exact)
  uint64_t RF;       // R 2^58 (exact)
  double R, v;
};
void build_zig(Zig* z);

// Kernel launchers (pmwa_kernels.cu).  All return a cudaError_t as int.
int upload_zig(const Zig& z);       // constants of pmwa_kernels.cu
int upload_zig_tile(const Zig& z);  // constants of pmwa_tile.cu
int upload_zig_green(const Zig& z); // constants of pmwa_green.cu
int launch_boundary(const Dev& d, int dir, void* stream);
int launch_temporal(const Dev& d, void* stream);  // Step 1, one warp per site
int launch_temporal_batch(const Dev* devs, const BatchBase* base, const int2* work, int n_work, int it, int cap,
                          void* stream);
int temporal_sites_per_block();
int prepare_temporal(int cap);
int launch_tile(const Dev& d, int stop, void* stream);
int tile_class(int domain_sites, int smem);
// batch launch groups: 3 CTA-size classes x residency levels by shared memory
constexpr int kResidencyLevels = 6;
constexpr int kBatchGroups = 4 * kResidencyLevels;
int launch_tile_batch(int cls, const Dev* devs, const BatchBase* base, const int2* work, int n_work, int smem,
                      int it, int stop, void* stream);
int launch_boundary_batch(const Dev* devs, const BatchBase* base, const int2* work, int n_work, int it, int dir,
                          int cap, void* stream);
int boundary_bonds_per_block(int cap);
int prepare_boundary(int cap);
int prepare_tile_batch(int cls, int smem);
int launch_advance(BatchBase* base, int n, int S, void* stream);
int launch_rho(const Dev& d, int K, double* out, void* stream);
// n Philox4x32-10 blocks: in[6 j ..] = c0..c3, k0, k1; out[4 j ..] = output
int launch_philox(const uint32_t* in, uint32_t* out, int64_t n, void* stream);
// Invariant check of the current configuration (codes as PMWA_CHECK_*):
// *out = ~0 when all hold, else min over failing sites of site << 4 | code.
int launch_check(const Dev& d, unsigned long long* out, void* stream);
// Supplement S-I estimators resolved by the component of Q (pmwa_green.cu)
constexpr int kMaxGreenSlices = 64;
int launch_rho_alpha(const Dev& d, int K, int s0, int ns, double* rho, int32_t* iv, void* stream);
int launch_green_tau(const Dev& d, int K, int rmax, double* rho, double* sums, void* stream);
constexpr int kMaxNpoint = 16;
int launch_npoint(int K, int n, int m, const double* rho, const int32_t* sites, double eta, double* out,
                  void* stream);
// component-resolved n-point functions of listed (site, slice, component)
// tuples at arbitrary times (pmwa_npoint_alpha)
int launch_npoint_alpha(const Dev& d, int K, int n, int m, const int32_t* pts, double* out, void* stream);
constexpr int kCheckNone = 0x7fffffff;
constexpr int kCheckCapacity = 1, kCheckTag = 2, kCheckOrder = 3, kCheckContinuity = 4, kCheckBase = 5,
              kCheckBond = 6, kCheckPartner = 7, kCheckConservation = 8;
int launch_green(int Lx, int Ly, int K, int rmax, const double* rho, double* sums, void* stream);
// rho slices through the library's own static device scratch (no allocation)
int rho_slices_static(const Dev& d, int K, double* host_out, void* stream);
// shared-memory plan of the tile kernel for this instance (fills the sm_*
// offsets); returns false if a domain cannot fit in shared memory.
bool plan_tile_smem(Dev* d, double legs_want, double cands_per_bond);

// Step-5 sub-block count along one axis (host copy of the device rule).
inline int sb_slots_host(int D, int B, int nd) {
  if (B == 0 || B >= D) return 1;
  return (nd == 1) ? D / B : D / B + 1;
}

}  // namespace pmwa
