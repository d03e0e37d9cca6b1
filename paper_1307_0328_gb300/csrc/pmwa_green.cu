// pmwa_green.cu -- Supplement S-I estimators resolved by the component of Q.
//
//   k_rho_alpha       rho_b and rho_b+ at K equal-time slices, one thread per site
//   k_green_tau_site  the two-point densities of one site (r = 0), one thread per site
//   k_green_tau_r     products of one-point densities of two sites (r >= 1)
//
// For X inside the interval I between two vertex legs of a site (p the state
// above the lower leg, q the state below the upper one, I1 the part of I
// below X, I2 the part above) the density of worms of type a at X is
//   rho_a(X) = eta <q| e^{I2 eta Q} Q_a e^{I1 eta Q} |p> / <q| e^{I eta Q} |p>,
// with Q_b = b taking 1 to 0 and Q_b+ = b+ taking 0 to 1.  One site's
// <a| e^{x Q} |b> is cosh x (a = b) or sinh x (a != b) = e^x F(a ^ b, x) / 2
// with F(0, x) = 2 + expm1(-2x) and F(1, x) = -expm1(-2x); the factors e^x
// cancel because I1 + I2 = I, counted in worm grid points (x = count beta eta
// / 2^59).  A site without vertex legs has no reference point on its circle:
// its density is the trace form eta Tr[Q_a e^{x Q}] / Tr[e^{x Q}] over the
// whole circle.  Two points on one interval take both operators inside the
// interval's matrix element; on two intervals the densities multiply.
//
// Every value is a fixed sequence of binary64 operations (no contraction), so
// the per-slice densities are reproducible bit for bit.
#include <cuda_runtime.h>

#include "pmwa_device.cuh"

namespace pmwa {

namespace {

constexpr uint32_t kCntMaskG = 0x7fffffffu;
constexpr uint64_t kMask62G = kTwo62 - 1;

struct SliceInfo {
  int iv;          // event index of the lower leg, -1: the site has no legs
  int p, q;        // state above the lower leg, below the upper one
  uint64_t M, M1;  // worm points of the interval, and below the slice
  uint64_t off;    // pk distance from the lower leg up to the slice
  uint64_t pt;     // the slice's pk
};

__device__ __forceinline__ uint64_t slice_pk(int K, int k) {
  const uint64_t q62 = kTwo62 / uint64_t(K), r62 = kTwo62 % uint64_t(K);
  return uint64_t(k) * q62 + (uint64_t(k) * r62) / uint64_t(K);
}

__device__ __forceinline__ double Fsig(int sigma, uint64_t M, double XW) {
  const double e = expm1_det(__dmul_rn(-2.0, __dmul_rn(__ull2double_rn(M), XW)));
  return sigma ? -e : __dadd_rn(2.0, e);
}
__device__ __forceinline__ int q_in(int a) { return 1 - a; }
__device__ __forceinline__ int q_out(int a) { return a; }

// the interval of the slice at pt on a site whose legs are known to exist
// (lo: the last leg with pk <= pt, or the last leg of the circle)
__device__ __forceinline__ void slice_at(const uint64_t* Kk, int n, int lo, uint64_t pt, SliceInfo* z) {
  int hi = lo;
  for (int i = 1; i <= n; ++i) { hi = (lo + i) % n; if (!kworm(Kk[hi])) break; }
  const uint64_t plo = kpk(Kk[lo]), phi = kpk(Kk[hi]);
  z->iv = lo;
  z->p = kab(Kk[lo]);
  z->q = kbl(Kk[hi]);
  z->M = wpts(plo, phi);
  z->M1 = (pt == plo) ? 0 : wpts(plo, pt);
  z->off = (pt - plo) & kMask62G;
  z->pt = pt;
}

// Walks the site's events and the K slices together, calling fn(k, z) for
// each slice in order.
template <class Fn>
__device__ __forceinline__ void for_slices(const Dev& d, int s, int K, Fn fn) {
  const uint64_t* Kk = d.keyA + size_t(s) * d.cap;
  const int n = min(int(d.cntA[s] & kCntMaskG), d.cap);
  int last = -1;
  for (int i = 0; i < n; ++i) if (!kworm(Kk[i])) last = i;
  SliceInfo z;
  if (last < 0) {
    for (int k = 0; k < K; ++k) {
      z.iv = -1; z.p = z.q = 0; z.M = kTwo59; z.M1 = 0; z.off = 0; z.pt = slice_pk(K, k);
      fn(k, z);
    }
    return;
  }
  int lo = last, i = 0;
  for (int k = 0; k < K; ++k) {
    const uint64_t pt = slice_pk(K, k);
    while (i < n && kpk(Kk[i]) <= pt) { if (!kworm(Kk[i])) lo = i; ++i; }
    slice_at(Kk, n, lo, pt, &z);
    fn(k, z);
  }
}

__device__ __forceinline__ double rho_one(const SliceInfo& z, int a, double eta, double XW) {
  if (z.iv < 0) return __dmul_rn(eta, __ddiv_rn(Fsig(1, kTwo59, XW), __dmul_rn(2.0, Fsig(0, kTwo59, XW))));
  const double num = __dmul_rn(Fsig(z.q ^ q_out(a), z.M - z.M1, XW), Fsig(q_in(a) ^ z.p, z.M1, XW));
  return __dmul_rn(eta, __ddiv_rn(num, __dmul_rn(2.0, Fsig(z.q ^ z.p, z.M, XW))));
}

// Q_a1 at slice z1 and Q_a2 at slice z2 of one interval of a site
__device__ __forceinline__ double rho_two_same(const SliceInfo& z1, int a1, const SliceInfo& z2, int a2, double eta,
                                               double XW) {
  const double eta2 = __dmul_rn(eta, eta);
  if (z1.iv < 0) {
    const uint64_t Ib = wpts(z1.pt, z2.pt), Ic = kTwo59 - Ib;
    const double num = __dmul_rn(Fsig(q_in(a2) ^ q_out(a1), Ib, XW), Fsig(q_in(a1) ^ q_out(a2), Ic, XW));
    return __dmul_rn(eta2, __ddiv_rn(num, __dmul_rn(4.0, Fsig(0, kTwo59, XW))));
  }
  const bool swap = z2.off < z1.off;
  const SliceInfo& L = swap ? z2 : z1;
  const SliceInfo& U = swap ? z1 : z2;
  const int aL = swap ? a2 : a1, aU = swap ? a1 : a2;
  const uint64_t Ia = L.M1, Ib = U.M1 - L.M1, Ic = L.M - U.M1;
  const double num = __dmul_rn(__dmul_rn(Fsig(L.q ^ q_out(aU), Ic, XW), Fsig(q_in(aU) ^ q_out(aL), Ib, XW)),
                               Fsig(q_in(aL) ^ L.p, Ia, XW));
  return __dmul_rn(eta2, __ddiv_rn(num, __dmul_rn(4.0, Fsig(L.q ^ L.p, L.M, XW))));
}

// sites s0 <= s < s0 + ns: rho[((s - s0) K + k) 2 + a]; iv[(s - s0) K + k]
// when iv is not null
__global__ void k_rho_alpha(const __grid_constant__ Dev d, int K, int s0, int ns, double* rho, int32_t* iv) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= ns) return;
  const int s = s0 + u;
  for_slices(d, s, K, [&](int k, const SliceInfo& z) {
    const size_t o = size_t(u) * K + k;
    rho[2 * o] = rho_one(z, 0, d.eta, d.XW);
    rho[2 * o + 1] = rho_one(z, 1, d.eta, d.XW);
    if (iv) iv[o] = z.iv;
  });
}

// the slice k of site s found by bisection (the same interval as the walk in
// for_slices): the last vertex leg with pk <= pt, else the last leg of the
// circle; `last` is the site's last vertex leg (-1: none)
__device__ __forceinline__ void slice_one(const uint64_t* Kk, int n, int last, int K, int k, SliceInfo* z) {
  const uint64_t pt = slice_pk(K, k);
  if (last < 0) { z->iv = -1; z->p = z->q = 0; z->M = kTwo59; z->M1 = 0; z->off = 0; z->pt = pt; return; }
  int a = 0, b = n;  // first event with pk > pt
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (kpk(Kk[mid]) <= pt) a = mid + 1; else b = mid;
  }
  int lo = last;
  for (int j = a - 1; j >= 0; --j) if (!kworm(Kk[j])) { lo = j; break; }
  slice_at(Kk, n, lo, pt, z);
}

// sums[dk] += sum over sites and slices k of the density of b+ at slice k and
// b at slice k + dk (mod K) on the same site, dk = 1..K-1
__global__ void k_green_tau_site(const __grid_constant__ Dev d, int K, double* sums) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = s < d.N;
  const uint64_t* Kk = act ? d.keyA + size_t(s) * d.cap : nullptr;
  const int n = act ? min(int(d.cntA[s] & kCntMaskG), d.cap) : 0;
  int last = -1;
  for (int i = 0; i < n; ++i) if (!kworm(Kk[i])) last = i;
  for (int dk = 1; dk < K; ++dk) {
    double acc = 0.0;
    if (act) {
      for (int k = 0; k < K; ++k) {
        SliceInfo z1, z2;
        slice_one(Kk, n, last, K, k, &z1);
        slice_one(Kk, n, last, K, (k + dk) % K, &z2);
        const double v = (z1.iv != z2.iv) ? __dmul_rn(rho_one(z1, 1, d.eta, d.XW), rho_one(z2, 0, d.eta, d.XW))
                                          : rho_two_same(z1, 1, z2, 0, d.eta, d.XW);
        acc = __dadd_rn(acc, v);
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(0xffffffffu, acc, o));
    if ((threadIdx.x & 31) == 0) atomicAdd(sums + dk, acc);
  }
}

// blockIdx.y = d rmax + r - 1 (d = 0: x, 1: y; r = 1..rmax), blockIdx.z = dk:
// sums[(d (rmax + 1) + r) K + dk] += sum_{i,k} rho_b(i + r e_d, k + dk) rho_b+(i, k)
__global__ void k_green_tau_r(int Lx, int Ly, int K, int rmax, const double* __restrict__ rho, double* sums) {
  const int N = Lx * Ly;
  const int dir = int(blockIdx.y) / rmax, r = int(blockIdx.y) % rmax + 1, dk = int(blockIdx.z);
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int x = i % Lx, y = i / Lx;
    const int j = dir == 0 ? (x + r) % Lx + Lx * y : x + Lx * ((y + r) % Ly);
    const double* ri = rho + size_t(i) * K * 2;
    const double* rj = rho + size_t(j) * K * 2;
    for (int k = 0; k < K; ++k) acc = __dadd_rn(acc, __dmul_rn(rj[2 * ((k + dk) % K)], ri[2 * k + 1]));
  }
  for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(0xffffffffu, acc, o));
  if ((threadIdx.x & 31) == 0) atomicAdd(sums + (size_t(dir) * (rmax + 1) + r) * K + dk, acc);
}

// Supplement S-I n-point functions of distinct sites at equal time: tuple j
// holds n sites (sites[j n + c]); out[j] = (sum_k prod_c rho[s_c K + k] / K)
// / eta^n, the product in tuple order from 1.0, the sum over the slices in
// order, eta^n by n multiplications from 1.0.  Distinct sites never share an
// interval, so the densities multiply.
__global__ void k_npoint(int K, int n, int m, const double* __restrict__ rho, const int32_t* __restrict__ sites,
                         double eta, double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int32_t* t = sites + size_t(j) * n;
  double acc = 0.0;
  for (int k = 0; k < K; ++k) {
    double p = 1.0;
    for (int c = 0; c < n; ++c) p = __dmul_rn(p, rho[size_t(t[c]) * K + k]);
    acc = __dadd_rn(acc, p);
  }
  double etan = 1.0;
  for (int c = 0; c < n; ++c) etan = __dmul_rn(etan, eta);
  out[j] = __ddiv_rn(__ddiv_rn(acc, double(K)), etan);
}

// Joint density of g operators Q_a[0..g) at the points z[idx[0..g)] of one
// interval, in time order (Supplement S-I with every operator inserted in the
// interval's matrix element):
//   eta^g <q| e^{I_g Q} Q_a[g-1] ... Q_a[0] e^{I_0 Q} |p> / <q| e^{I Q} |p>
//     = eta^g F(in_a[0] ^ p, I_0) prod_j F(in_a[j] ^ out_a[j-1], I_j) F(q ^ out_a[g-1], I_g)
//       / (2^g F(q ^ p, I)),
// I_0 the worm points below the first point, I_j between points j-1 and j,
// I_g above the last; on a site without legs the cyclic trace
//   eta^g prod_j F(in_a[j+1] ^ out_a[j], I_j) / (2^g F(0, 2^59)),
// I_j between points j and j + 1 and the last piece closing the circle.
__device__ double rho_interval(const SliceInfo* z, const int* idx, const int* a, int g, double eta, double XW) {
  double num = 1.0, etag = 1.0, den = 1.0;
  for (int j = 0; j < g; ++j) { etag = __dmul_rn(etag, eta); den = __dmul_rn(den, 2.0); }
  const SliceInfo& z0 = z[idx[0]];
  if (z0.iv < 0) {
    uint64_t used = 0;
    for (int j = 0; j < g; ++j) {
      const int nx = (j + 1) % g;
      const uint64_t piece = (j + 1 < g) ? wpts(z[idx[j]].pt, z[idx[j + 1]].pt) : kTwo59 - used;
      used += piece;
      num = __dmul_rn(num, Fsig(q_in(a[nx]) ^ q_out(a[j]), piece, XW));
    }
    return __dmul_rn(etag, __ddiv_rn(num, __dmul_rn(den, Fsig(0, kTwo59, XW))));
  }
  num = Fsig(q_in(a[0]) ^ z0.p, z[idx[0]].M1, XW);
  for (int j = 1; j < g; ++j)
    num = __dmul_rn(num, Fsig(q_in(a[j]) ^ q_out(a[j - 1]), z[idx[j]].M1 - z[idx[j - 1]].M1, XW));
  num = __dmul_rn(num, Fsig(z0.q ^ q_out(a[g - 1]), z0.M - z[idx[g - 1]].M1, XW));
  return __dmul_rn(etag, __ddiv_rn(num, __dmul_rn(den, Fsig(z0.q ^ z0.p, z0.M, XW))));
}

// Supplement S-I n-point functions resolved by the component of Q at
// arbitrary times: tuple j holds n points (site, slice, component) at
// pts[(j n + c) 3 ..]; out[j] = (sum over the K cyclic shifts of the slices of
// the product over intervals of the joint density of their points) / K /
// eta^n.  The points are grouped by interval (site and lower vertex leg, or
// the whole circle of a site without legs) in order of first appearance, each
// group's points in time order (insertion sort by the offset from the lower
// leg, or by time point on a site without legs).
__global__ void k_npoint_alpha(const __grid_constant__ Dev d, int K, int n, int m, const int32_t* __restrict__ pts,
                               double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int32_t* t = pts + size_t(j) * size_t(n) * 3;
  int last[kMaxNpoint], cnt[kMaxNpoint];
  for (int c = 0; c < n; ++c) {
    const uint64_t* Kk = d.keyA + size_t(t[3 * c]) * d.cap;
    cnt[c] = min(int(d.cntA[t[3 * c]] & kCntMaskG), d.cap);
    last[c] = -1;
    for (int i = 0; i < cnt[c]; ++i) if (!kworm(Kk[i])) last[c] = i;
  }
  double acc = 0.0;
  for (int sh = 0; sh < K; ++sh) {
    SliceInfo z[kMaxNpoint];
    for (int c = 0; c < n; ++c)
      slice_one(d.keyA + size_t(t[3 * c]) * d.cap, cnt[c], last[c], K, (t[3 * c + 1] + sh) % K, &z[c]);
    unsigned done = 0;
    double prod = 1.0;
    for (int c = 0; c < n; ++c) {
      if (done & (1u << c)) continue;
      int idx[kMaxNpoint], a[kMaxNpoint], g = 0;
      for (int e = c; e < n; ++e)
        if (!(done & (1u << e)) && t[3 * e] == t[3 * c] && z[e].iv == z[c].iv) { idx[g++] = e; done |= 1u << e; }
      const bool ring = z[c].iv < 0;
      for (int i = 1; i < g; ++i)
        for (int k = i; k > 0; --k) {
          const uint64_t ka = ring ? z[idx[k]].pt : z[idx[k]].off, kb = ring ? z[idx[k - 1]].pt : z[idx[k - 1]].off;
          if (ka < kb) { const int tmp = idx[k]; idx[k] = idx[k - 1]; idx[k - 1] = tmp; } else break;
        }
      for (int i = 0; i < g; ++i) a[i] = t[3 * idx[i] + 2];
      prod = __dmul_rn(prod, rho_interval(z, idx, a, g, d.eta, d.XW));
    }
    acc = __dadd_rn(acc, prod);
  }
  double etan = 1.0;
  for (int c = 0; c < n; ++c) etan = __dmul_rn(etan, d.eta);
  out[j] = __ddiv_rn(__ddiv_rn(acc, double(K)), etan);
}

}  // namespace

int launch_npoint_alpha(const Dev& d, int K, int n, int m, const int32_t* pts, double* out, void* stream) {
  if (m <= 0) return 0;
  k_npoint_alpha<<<(m + 63) / 64, 64, 0, cudaStream_t(stream)>>>(d, K, n, m, pts, out);
  return int(cudaGetLastError());
}

int launch_npoint(int K, int n, int m, const double* rho, const int32_t* sites, double eta, double* out,
                  void* stream) {
  if (m <= 0) return 0;
  k_npoint<<<(m + 127) / 128, 128, 0, cudaStream_t(stream)>>>(K, n, m, rho, sites, eta, out);
  return int(cudaGetLastError());
}

// this translation unit's copy of the constant tables (expm1_det reads them)
int upload_zig_green(const Zig& z) { return upload_constants(z); }

int launch_rho_alpha(const Dev& d, int K, int s0, int ns, double* rho, int32_t* iv, void* stream) {
  k_rho_alpha<<<(ns + 127) / 128, 128, 0, cudaStream_t(stream)>>>(d, K, s0, ns, rho, iv);
  return int(cudaGetLastError());
}

int launch_green_tau(const Dev& d, int K, int rmax, double* rho, double* sums, void* stream) {
  cudaStream_t st = cudaStream_t(stream);
  const size_t nsum = size_t(2) * size_t(rmax + 1) * size_t(K);
  if (cudaMemsetAsync(sums, 0, nsum * sizeof(double), st) != cudaSuccess) return int(cudaGetLastError());
  k_green_tau_site<<<(d.N + 127) / 128, 128, 0, st>>>(d, K, sums);
  if (cudaGetLastError() != cudaSuccess) return PMWA_ECUDA;
  if (rmax > 0) {
    k_rho_alpha<<<(d.N + 127) / 128, 128, 0, st>>>(d, K, 0, d.N, rho, nullptr);
    if (cudaGetLastError() != cudaSuccess) return PMWA_ECUDA;
    const int bx = d.N < 256 * 152 ? (d.N + 255) / 256 : 152;
    k_green_tau_r<<<dim3(bx, 2 * rmax, K), 256, 0, st>>>(d.Lx, d.Ly, K, rmax, rho, sums);
  }
  return int(cudaGetLastError());
}

}  // namespace pmwa
