// Host set-up of a problem: operator coefficients, the spectrum rectangle (§3 Lemma 3.1),
// the contour nodes and weights (§6.1, §6.2 eq:quad-points, eq:quad-radius) and the
// parameters of the polynomial scheme at every node (§4.2 eq:fix-pt-conv).
//
// Readings used where the paper leaves the procedure open:
//  * the rectangle is B = [b1, b2] x [-rho2, 0] with exact Weyl bounds of s L_h - diag(m)
//    (the 7-point Dirichlet and the Fourier spectral eigenvalues are known in closed form)
//    and rho2 = max a;
//  * delta has the sign of Im z_j; |delta| is searched on 512 equal steps of
//    (0, 4(q+1)/W], W = max |lambda - z0| over the sampled boundary of B, then refined by
//    golden-section search on the bracket of the best grid point;
//  * each side of B is sampled at 256 equally spaced points (4 * 256 points in all);
//  * sweeps = ceil(ln(reduction) / -ln(nu)); the order q with the fewest matrix-vector
//    products q*sweeps wins, ties to the smaller q.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "hz_internal.h"

namespace hz {
namespace {

struct cplx {
  double re, im;
};
inline cplx operator+(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
inline cplx operator-(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
inline cplx operator*(cplx a, cplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
inline cplx operator/(cplx a, double d) { return {a.re / d, a.im / d}; }
inline double cabs(cplx a) { return std::hypot(a.re, a.im); }

constexpr double kPi = 3.14159265358979323846;

// Taylor sum 1 + u + u^2/2! + ... + u^q/q! with u = -i delta (lambda - z0) (eq:exp-taylor).
double ptilde_abs(cplx lam, int q, double delta, cplx z0) {
  const cplx d = lam - z0;
  const cplx u = {delta * d.im, -delta * d.re};  // -i * delta * d
  cplx term = {1.0, 0.0}, total = {1.0, 0.0};
  for (int j = 1; j <= q; ++j) {
    term = (term * u) / double(j);
    total = total + term;
  }
  return cabs(total);
}

// Rate max_{boundary} |ptilde(lam)| / |ptilde(z)| of one (q, delta).
double rate(int q, double delta, cplx z, cplx z0, const std::vector<cplx>& bd) {
  double mx = 0.0;
  for (const cplx& l : bd) mx = std::max(mx, ptilde_abs(l, q, delta, z0));
  return mx / ptilde_abs(z, q, delta, z0);
}

std::vector<cplx> boundary(double b1, double b2, double rho2, int per_side) {
  const cplx v[4] = {{b1, 0.0}, {b2, 0.0}, {b2, -rho2}, {b1, -rho2}};
  std::vector<cplx> pts;
  pts.reserve(4 * per_side);
  for (int side = 0; side < 4; ++side) {
    const cplx a = v[side], b = v[(side + 1) % 4];
    for (int t = 0; t < per_side; ++t) {
      const double tt = double(t) / per_side;
      pts.push_back(a + (b - a) * cplx{tt, 0.0});
    }
  }
  return pts;
}

// Best delta for one order q: grid then golden section; returns (delta, nu).
void best_delta(int q, cplx z, cplx z0, const std::vector<cplx>& bd, double& delta_out,
                double& nu_out) {
  const int ngrid = 512;
  const double tol = 1e-10;
  const double sgn = z.im > 0 ? 1.0 : -1.0;
  double W = 0.0;
  for (const cplx& l : bd) W = std::max(W, cabs(l - z0));
  const double dmax = 4.0 * (q + 1) / W;
  int kbest = 0;
  double vbest = 0.0;
  std::vector<double> grid(ngrid);
  for (int k = 0; k < ngrid; ++k) {
    grid[k] = dmax * double(k + 1) / ngrid;
    const double v = rate(q, sgn * grid[k], z, z0, bd);
    if (k == 0 || v < vbest) {
      vbest = v;
      kbest = k;
    }
  }
  double a = kbest > 0 ? grid[kbest - 1] : 0.0;
  double b = kbest + 1 < ngrid ? grid[kbest + 1] : dmax;
  const double g = (std::sqrt(5.0) - 1.0) / 2.0;
  double c = b - g * (b - a), d = a + g * (b - a);
  double fc = rate(q, sgn * c, z, z0, bd), fd = rate(q, sgn * d, z, z0, bd);
  while (b - a > tol * dmax) {
    if (fc < fd) {
      b = d;
      d = c;
      fd = fc;
      c = b - g * (b - a);
      fc = rate(q, sgn * c, z, z0, bd);
    } else {
      a = c;
      c = d;
      fc = fd;
      d = a + g * (b - a);
      fd = rate(q, sgn * d, z, z0, bd);
    }
  }
  double best = 0.5 * (a + b);
  double nbest = rate(q, sgn * best, z, z0, bd);
  if (vbest < nbest) {
    best = grid[kbest];
    nbest = vbest;
  }
  delta_out = sgn * best;
  nu_out = nbest;
}

}  // namespace

void setup_operator(const hz_grid& g, const double* c, Setup& out) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  double cmin = c[0];
  for (long long p = 1; p < n; ++p) cmin = std::min(cmin, c[p]);
  out.c_min = cmin;
  out.s = cmin * cmin / (g.omega * g.omega);
  out.m.resize(n);
  double mmax = 0.0, mmin = 0.0, amax = 0.0;
  const int L = g.layer_cells;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const long long p = i + (long long)g.nx * (j + (long long)g.ny * k);
        const double mp = (cmin * cmin) / (c[p] * c[p]);
        out.m[p] = mp;
        if (p == 0 || mp > mmax) mmax = mp;
        if (p == 0 || mp < mmin) mmin = mp;
        if (L > 0) {
          auto dep = [L](int idx, int nn) { return std::max(0, L - std::min(idx, nn - 1 - idx)); };
          const int d = std::max(dep(i, g.nx), std::max(dep(j, g.ny), dep(k, g.nz)));
          const double t = double(d) / double(L);
          amax = std::max(amax, (g.sigma_max * (t * t)) * mp);
        }
      }
  double lo = 0.0, hi = 0.0;
  const int dims[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < 3; ++a) {
    const double nn = dims[a];
    if (g.discretization == HZ_DISC_SPECTRAL) {
      // Fourier spectral -Delta (eq:eig-Laplacian-spectral): the constant mode gives 0, the
      // largest wavenumber along an axis of n points is 2 pi floor(n/2) / (n h)
      const double k = 2.0 * kPi * std::floor(nn / 2.0) / (nn * g.h);
      hi += k * k;
    } else {
      // extreme eigenvalues of the Dirichlet -Delta_h: sums over the axes of
      // (4/h^2) sin^2(k pi / (2(n+1))) at k = 1 and k = n
      const double s1 = std::sin(kPi / (2.0 * (nn + 1.0)));
      const double s2 = std::sin(nn * kPi / (2.0 * (nn + 1.0)));
      lo += 4.0 / (g.h * g.h) * s1 * s1;
      hi += 4.0 / (g.h * g.h) * s2 * s2;
    }
  }
  out.b1 = out.s * lo - mmax;
  out.b2 = out.s * hi - mmin;
  out.rho2 = amax;
}

bool setup_nodes(const Setup& su, const hz_contour_opts& co, std::vector<NodeParams>& nodes,
                 std::string& err) {
  const int J = co.J;
  const double phi = kPi / J;
  const double r = (su.rho2 / 2.0 + co.eps) / std::sin(phi);
  const double cre = -co.t * r * std::cos(phi), cim = -su.rho2 / 2.0;
  const std::vector<cplx> bd = boundary(su.b1, su.b2, su.rho2, 256);
  nodes.assign(J, NodeParams{});
  for (int jn = 0; jn < J; ++jn) {
    const double th = phi + 2.0 * kPi * jn / J;  // (2j-1) phi for j = jn+1
    NodeParams& nd = nodes[jn];
    nd.zr = cre + co.t * r * std::cos(th);
    nd.zi = cim + r * std::sin(th);
    nd.sr = r * std::cos(th) / J;
    nd.si = co.t * r * std::sin(th) / J;
    nd.z0r = 0.5 * (su.b1 + su.b2);
    nd.z0i = nd.zi;
    const cplx z = {nd.zr, nd.zi}, z0 = {nd.z0r, nd.z0i};
    int best_cost = -1;
    for (int q = 1; q <= co.qmax; ++q) {
      double delta, nu;
      best_delta(q, z, z0, bd, delta, nu);
      if (!(nu < 1.0)) continue;
      const int sw = std::max(1, int(std::ceil(std::log(co.reduction) / -std::log(nu))));
      const int cost = q * sw;
      if (best_cost < 0 || cost < best_cost) {
        best_cost = cost;
        nd.q = q;
        nd.delta = delta;
        nd.nu = nu;
        nd.sweeps = sw;
      }
    }
    if (best_cost < 0) {
      err = "no polynomial order <= qmax converges at node " + std::to_string(jn);
      return false;
    }
  }
  return true;
}

}  // namespace hz
