// pmwa_obs.cpp -- Step 6 of the pseudo code turned into physical observables:
// energy, density, order parameter (raw and Supplement S-I estimator) and
// kinetic term per measured sweep, their means with binned errors, the
// worms-per-domain figures, and the N_cycle rule.  Host code only: it reads
// the rows that pmwa_measure hands out.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/pmwa.h"

namespace {

struct Model {
  double N, Nb, C, d_mean, beta, eta, t;
  double domains;
};

// Eq. 5 per bond: E(na, nb) = V na nb - (mu/4)(na + nb); C = max E + c_off
// (c_off < 0 means t/2); d(s) = C - E(s).
bool model_of(const pmwa_params* p, Model* m) {
  if (!p || pmwa_footprint(p) == 0) return false;
  const double c_off = (p->c_off < 0.0) ? 0.5 * p->t : p->c_off;
  double E[4], Emax = -INFINITY;
  for (int s = 0; s < 4; ++s) {
    const int na = s & 1, nb = s >> 1;
    E[s] = p->V * double(na * nb) - (p->mu / 4.0) * double(na + nb);
    Emax = std::max(Emax, E[s]);
  }
  m->C = Emax + c_off;
  double sum = 0.0;
  for (int s = 0; s < 4; ++s) sum += m->C - E[s];
  m->d_mean = sum / 4.0;
  m->N = double(p->Lx) * double(p->Ly);
  m->Nb = 2.0 * m->N;
  m->beta = p->beta;
  m->eta = p->eta;
  m->t = p->t;
  const int dx = p->dom_x ? p->dom_x : p->Lx, dy = p->dom_y ? p->dom_y : p->Ly;
  const int nt = p->dom_tau > 1 ? p->dom_tau : 1;
  m->domains = double(p->Lx / dx) * double(p->Ly / dy) * double(nt);
  return true;
}

void series_of(const Model& m, const pmwa_row& r, double* o) {
  const double occ = double(r.occ_lo) + double(r.occ_hi) * 0x1p64;
  const double E = (m.Nb * m.C - double(r.n_v) / m.beta) / m.N;
  const double q_impr = r.q_impr / (m.beta * m.eta * m.N);
  o[PMWA_S_E] = E;
  o[PMWA_S_E_ETA] = E - m.eta * q_impr;
  o[PMWA_S_N] = occ / (0x1p62 * m.N);
  o[PMWA_S_Q_RAW] = double(r.n_w) / (m.beta * m.eta * m.N);
  o[PMWA_S_Q_IMPR] = q_impr;
  o[PMWA_S_KIN] = (m.t > 0.0) ? double(r.n_k) / (m.beta * m.t * m.Nb) : 0.0;
}

}  // namespace

extern "C" {

int pmwa_row_observables(const pmwa_params* p, const pmwa_row* rows, int64_t n_rows, double* out) {
  Model m;
  if (!model_of(p, &m) || n_rows < 0 || (n_rows && (!rows || !out))) return PMWA_EINVAL;
  for (int64_t r = 0; r < n_rows; ++r) series_of(m, rows[r], out + r * PMWA_SERIES);
  return PMWA_OK;
}

int pmwa_observables(const pmwa_params* p, const pmwa_row* rows, int64_t n_rows, int32_t bins, pmwa_obs* out) {
  Model m;
  if (!model_of(p, &m) || !out || !rows || bins < 2 || n_rows < bins) return PMWA_EINVAL;
  const int64_t per = n_rows / bins, used = per * bins;
  // bin means of each series, then the mean and the standard error over bins
  double mean[PMWA_SERIES] = {}, sq[PMWA_SERIES] = {};
  std::vector<double> bm(size_t(bins) * PMWA_SERIES, 0.0);
  double nv = 0.0, nw = 0.0, wmin = INFINITY, empty = 0.0;
  for (int32_t b = 0; b < bins; ++b) {
    for (int64_t r = b * per; r < (b + 1) * per; ++r) {
      double o[PMWA_SERIES];
      series_of(m, rows[r], o);
      for (int k = 0; k < PMWA_SERIES; ++k) bm[size_t(b) * PMWA_SERIES + k] += o[k];
      nv += double(rows[r].n_v);
      nw += double(rows[r].n_w);
      wmin = std::min(wmin, double(rows[r].w_dom_min));
      empty += double(rows[r].dom_empty);
    }
    for (int k = 0; k < PMWA_SERIES; ++k) {
      bm[size_t(b) * PMWA_SERIES + k] /= double(per);
      mean[k] += bm[size_t(b) * PMWA_SERIES + k];
    }
  }
  for (int k = 0; k < PMWA_SERIES; ++k) mean[k] /= double(bins);
  for (int32_t b = 0; b < bins; ++b)
    for (int k = 0; k < PMWA_SERIES; ++k) {
      const double d = bm[size_t(b) * PMWA_SERIES + k] - mean[k];
      sq[k] += d * d;
    }
  double err[PMWA_SERIES];
  for (int k = 0; k < PMWA_SERIES; ++k) err[k] = std::sqrt(sq[k] / (double(bins) * double(bins - 1)));
  out->rows = used;
  out->bins = bins;
  out->pad = 0;
  out->E = mean[PMWA_S_E]; out->E_err = err[PMWA_S_E];
  out->E_eta = mean[PMWA_S_E_ETA]; out->E_eta_err = err[PMWA_S_E_ETA];
  out->n = mean[PMWA_S_N]; out->n_err = err[PMWA_S_N];
  out->Q_raw = mean[PMWA_S_Q_RAW]; out->Q_raw_err = err[PMWA_S_Q_RAW];
  out->Q_impr = mean[PMWA_S_Q_IMPR]; out->Q_impr_err = err[PMWA_S_Q_IMPR];
  out->kin = mean[PMWA_S_KIN]; out->kin_err = err[PMWA_S_KIN];
  out->n_v = nv / double(used);
  out->n_w = nw / double(used);
  out->w_dom_mean = out->n_w / m.domains;
  out->w_dom_min = wmin;
  out->dom_empty_frac = empty / (double(used) * m.domains);
  return PMWA_OK;
}

int pmwa_n_cycle(const pmwa_params* p, const pmwa_row* rows, int64_t n_rows, int32_t* n_cycle) {
  Model m;
  if (!model_of(p, &m) || !n_cycle || n_rows < 0 || (n_rows && !rows)) return PMWA_EINVAL;
  double nv, nw;
  if (n_rows > 0) {
    nv = 0.0;
    nw = 0.0;
    for (int64_t r = 0; r < n_rows; ++r) {
      nv += double(rows[r].n_v);
      nw += double(rows[r].n_w);
    }
    nv /= double(n_rows);
    nw /= double(n_rows);
  } else {
    nv = m.Nb * m.beta * (m.d_mean + m.t / 2.0);
    nw = m.beta * m.eta * m.N / 2.0;
  }
  const double c = std::ceil(2.0 * nv / std::max(nw, 1.0));
  *n_cycle = int32_t(std::max(1.0, std::min(512.0, c)));
  return PMWA_OK;
}

}  // extern "C"
