/*
 * clv_cooperfrye.c -- plain FP64 CPU oracle of the smooth Cooper-Frye
 * spectra.  TEST INFRASTRUCTURE ONLY, under the same rules as clv_oracle.c:
 * only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it, and it shares no code with the CUDA library.
 *
 * What it computes (Sec. 4, Eqs. (cooper_frye) and (feq)): the invariant
 * momentum distribution of one hadron species,
 *   dN/(dY pT dpT dphi) = g / (2 pi)^3  sum over surface elements of
 *                         p^mu dSigma_mu f_eq (1 + delta f),
 *   f_eq    = 1 / (exp[(p.u - mu)/T_f] + s),  s = +1 Fermi-Dirac, -1 Bose-Einstein,
 *                                               0 Boltzmann,
 *   delta f = (1 - s f_eq) p_mu p_nu pi^{mu nu} / (2 T_f^2 (eps + P)),
 * evaluated at the points of a (Y, pT, phi) grid (the paper uses 41 x 15 x 48
 * points, pT and phi at Gauss quadrature nodes).  Readings (C1-C4):
 *   C1 The surface is a list of elements (the finder's records: dSigma_mu
 *      covariant in (tau, x, y, eta_s), the position, u~ and pi~); the sum
 *      keeps the elements where p^mu dSigma_mu < 0, as the integral is
 *      written.
 *   C2 Milne momentum at the element's eta_s: p^tau = mT cosh(Y - eta_s),
 *      p^x = pT cos phi, p^y = pT sin phi, tau p^eta = mT sinh(Y - eta_s);
 *      so p^mu dSigma_mu = p^tau dSigma_tau + p^x dSigma_x + p^y dSigma_y +
 *      (tau p^eta / tau) dSigma_eta, and p.u = p~^tau u~^tau - p^x u~^x -
 *      p^y u~^y - p~^eta u~^eta with the tilde components.
 *   C3 p_mu p_nu pi^{mu nu} contracts p~_mu = (p~^tau, -p^x, -p^y, -p~^eta)
 *      with pi~ (the tilde metric diag(1, -1, -1, -1)).
 *   C4 Units: dSigma in fm^3 (dSigma_eta in fm^4), momenta in GeV; the sum
 *      is divided by (hbar c)^3, so the result is in GeV^-2.  eps + P is the
 *      equation of state's value at the freeze-out (an input).
 *
 * Pins (tests/test_oracle_cooperfrye.py): the boost-invariant tau = const
 * surface against the Bessel-function closed form, the momentum integral of
 * one element against n u.dSigma with n from Eq. (thermal_density_i), and
 * the pi moments against one-dimensional quadratures.
 */
#include <math.h>
#include <stdint.h>

#ifndef PLANT
#define PLANT 0
#endif

#define CF_HBARC 0.1973269804
#define CF_NREC 22

typedef struct {
  double mass;   /* GeV */
  double g;      /* degeneracy */
  int stat;      /* +1 Fermi-Dirac, -1 Bose-Einstein, 0 Boltzmann */
  double mu;     /* chemical potential, GeV */
  double Tf;     /* freeze-out temperature, GeV */
  double ePf;    /* eps + P at freeze-out, GeV/fm^3 */
  int viscous;   /* 1: delta f from pi~ */
} orc_cf_species;

/* pi~ component order: tt tx ty te xx xy xe yy ye ee */
static const int CF_PI[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};

/* the summand of one element at momentum (Y, pT, phi) */
static double cf_term(const orc_cf_species* sp, const double* r, double Y, double mT, double px, double py) {
  double tau = r[4], eta = r[7];
  double pt_ = mT * cosh(Y - eta);        /* p^tau */
  double pe_ = mT * sinh(Y - eta);        /* tau p^eta */
  double pdS = pt_ * r[0] + px * r[1] + py * r[2] + ((PLANT == 13) ? pe_ * tau : pe_ / tau) * r[3];
  double pu = pt_ * r[8] - px * r[9] - py * r[10] + ((PLANT == 15) ? 1.0 : -1.0) * pe_ * r[11];
  double f = 1.0 / (exp((pu - sp->mu) / sp->Tf) + ((PLANT == 14) ? -1.0 : 1.0) * (double)sp->stat);
  double df = 0.0;
  if (sp->viscous) {
    double pl[4] = {pt_, -px, -py, -pe_};
    double s = 0.0;
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) s += pl[m] * pl[n] * r[12 + CF_PI[m][n]];
    df = (1.0 - (double)sp->stat * f) * s / (2.0 * sp->Tf * sp->Tf * sp->ePf);
  }
  return pdS * f * (1.0 + df);
}

/* dN/(dY pT dpT dphi) at every (Y[a], pT[b], phi[c]) into out[(a*npt + b)*nphi + c]
 * from the nel element records (22 doubles each).  With absolute != 0 the
 * sum of the magnitudes of the summands instead (the scale that bounds the
 * rounding error of any summation order).  Returns 0, or -1 for a bad
 * argument. */
int orc_cooper_frye(const orc_cf_species* sp, const double* rec, int64_t nel, const double* Y, int nY,
                    const double* pT, int npt, const double* phi, int nphi, int absolute, double* out) {
  if (!(sp->Tf > 0) || nY < 0 || npt < 0 || nphi < 0 || nel < 0) return -1;
  if (sp->viscous && !(sp->ePf > 0)) return -1;
  const double norm = sp->g / pow(2.0 * M_PI * CF_HBARC, 3);
  long npts = (long)nY * npt * nphi;
#pragma omp parallel for schedule(dynamic, 4)
  for (long q = 0; q < npts; ++q) {
    int a = (int)(q / ((long)npt * nphi)), b = (int)((q / nphi) % npt), c = (int)(q % nphi);
    double mT = sqrt(pT[b] * pT[b] + sp->mass * sp->mass);
    double px = pT[b] * cos(phi[c]), py = pT[b] * sin(phi[c]);
    double s = 0.0;
    for (int64_t e = 0; e < nel; ++e) {
      double t = cf_term(sp, rec + e * CF_NREC, Y[a], mT, px, py);
      s += absolute ? fabs(t) : t;
    }
    out[q] = norm * s;
  }
  return 0;
}
