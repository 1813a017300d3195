// SIDM scattering-step ORACLE -- test infrastructure only.
//
// A plain, slow, FP64 CPU restatement of the Monte-Carlo self-interacting
// dark matter scattering step of Zier et al., "A Novel Implementation of
// Self-Interacting Dark Matter in AREPO-2" (Sec. 4).  It exists so that the
// CUDA path can be checked against it; only the test-suite, the smoke check
// and the benchmark's CPU-baseline leg may load it.  It shares no code with
// the CUDA library: its own neighbour search (a k-d tree, plus a brute-force
// mode), its own Philox generator written from Salmon et al. (SC'11), its own
// kernel, probability, draw and kick arithmetic.
//
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -fno-fast-math -shared -fPIC
// (no FMA contraction: every floating-point operation below is one IEEE
// round-to-nearest operation, in the order written).
//
// What each function follows:
//   philox4x32_10          Salmon, Moraes, Dror & Shaw (SC'11), Philox-4x32 with
//                          10 rounds (multipliers, Weyl key schedule, S-box).
//   separation_r2          minimum-image squared separation (periodic box) or
//                          plain squared separation (open boundaries).
//   count_within           neighbour count c_i(h) over all particles, active
//                          and inactive (Sec. 4.3, Fig. 3 caption).
//   bisect_h               h_SI found by bisection to N_ngb +- tol (Sec. 4.2,
//                          Sec. 4.5 "32 +- 5 neighbours").
//   kernel_w               cubic spline W_CS(q, h) (Sec. 4.2) and top-hat
//                          W_TH (Sec. 4.2), h = radius of compact support.
//   sigma_over_m           constant sigma/m, a table interpolated linearly in
//                          log v (Sec. 4.1), or the Yukawa-like
//                          sigma0/m / (1 + (v/w)^2)^2 (Sec. 5.2).
//   directed_probability   P(i|j) = 1/2 m_j (sigma/m) |v_i - v_j| W(r_ij, h_i) dt_i
//                          (Eqs. 10, 11 with the one-sided estimator, Eq. 14).
//   isotropic_direction    unit vector uniform on the sphere (Sec. 4.1),
//                          by Marsaglia's (1972) rejection method.
//   kick                   centre-of-momentum kick with outgoing relative speed
//                          eps |v_i - v_j| (Sec. 4.1; eps = 1: elastic).
//   step                   one scattering step for the active set, pairs drawn
//                          once, applied in a canonical order, and the per-pair
//                          timestep criterion (Eq. 18).
//
// Readings of points the paper leaves open (each is one deterministic choice):
//   * the neighbour count excludes the particle itself and uses r < h;
//   * bisection starts from h0 = L_ext * 2^-e with the largest e >= 0 such
//     that 8^e * N_ngb <= 4 N (about the mean-density radius of N_ngb
//     particles, exactly representable), doubles h while the count is too
//     small and no upper bracket is known, otherwise halves the bracket;
//     at most 128 evaluations, after which the last h is kept and a
//     non-convergence is counted;
//   * each unordered pair {i,j} is drawn ONCE against
//     P_pair = P(i|j)[i active, j in N(i)] + P(j|i)[j active, i in N(j)]
//     (the paper visits a pair from both sides with the factor 1/2 in each;
//     the expected number of scatters is the same while P_pair <= 1);
//   * acceptance uses start-of-step velocities; the kicks of accepted pairs
//     are applied one after another in ascending (ord, a, b) order, each
//     reading the current velocities (multiple scatters, Sec. 4.4);
//   * the random stream is Philox-4x32-10, key = (seed_lo, seed_hi),
//     counter = (step_lo, stream, a, b) with a = min id, b = max id;
//     stream 0 decides the pair, streams 1.. feed the direction rejection loop
//     (at most 64 tries, then e = (0,0,1) and a failure is counted);
//   * P_pair >= 1 is accepted (always) and counted;
//   * (v sigma/m)_max of Eq. 18 is taken over N(i) with start-of-step velocities.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

typedef struct {
  int n_ngb;        // target neighbour number N_ngb
  int ngb_tol;      // accepted band N_ngb +- ngb_tol
  double c_sidm;    // C_SIDM of Eq. 18
  double box;       // > 0: periodic cube side; 0: open boundaries
  int kernel;       // 0 cubic spline, 1 top-hat
  double fixed_h;   // > 0: every active particle uses this h (no bisection)
  int use_tree;     // 1: k-d tree neighbour search; 0: brute force O(N^2)
  int n_threads;    // OpenMP threads for the per-particle phases (0 = default)
  // estimator of g_ij: 0 one-sided W(r_ij, h_i) (Eq. 14); 1 kernel overlap
  // (Eq. 15, Appendix A) from the table ghat(a, s), a = min(h_i, h_j) / H,
  // s = r_ij / H, H = h_i + h_j: (ov_na + 1) x (ov_ns + 1) values on
  // a = k / (2 ov_na), s = l / ov_ns, row-major in a
  int estimator;
  int ov_na, ov_ns;
  const double* ov_table;
} orc_config;

typedef struct {
  int kind;         // 0 constant sigma/m; 1 Yukawa-like sigma0/m / (1+(v/w)^2)^2
  double sigma0;    // sigma0/m
  double w;         // velocity scale of the Yukawa-like law
  double inelastic; // 1 - eps: the outgoing relative speed is eps times the
                    // incoming one (Sec. 4.1); 0 = elastic, the paper's runs
  // kind 2: tabulated sigma/m(v) (Sec. 4.1), n >= 2 nodes, v increasing
  int32_t tab_n;
  const double* tab_v;
  const double* tab_s;
} orc_sigma;

typedef struct {
  int64_t n_active, n_candidate_pairs, n_accepted, n_p_ge_1, n_h_nonconv, n_dir_fail;
  double e_before, e_after, p_before[3], p_after[3];
  double sum_p;     // sum of P_pair over all candidate pairs
} orc_stats;

}  // extern "C"

namespace {

// ------------------------------------------------------------- Philox ---
// Philox-4x32 (Salmon et al., SC'11): a 4-word counter, a 2-word key, rounds
// of two 32x32->64 multiplies whose high halves are mixed with the other two
// counter words and the key; the key is bumped by the Weyl constants between
// rounds.
const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

void philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    const uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    const uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t y0 = hi1 ^ x1 ^ k0;
    const uint32_t y2 = hi0 ^ x3 ^ k1;
    x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void draw_words(uint64_t seed, uint64_t step, uint32_t stream, uint32_t a, uint32_t b,
                uint32_t w[4]) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const uint32_t ctr[4] = {(uint32_t)step, stream, a, b};
  philox4x32_10(key, ctr, w);
}

// 53-bit uniform in [0, 1) from two words, exact in FP64.
double uniform53(uint32_t wa, uint32_t wb) {
  const double hi = (double)(wa >> 5);   // 27 bits
  const double lo = (double)(wb >> 6);   // 26 bits
  return (hi * 67108864.0 + lo) * 0x1.0p-53;
}

// -------------------------------------------------------- geometry ---
struct Cloud {
  int64_t n;
  const double* pos;   // n x 3
  double box;
};

double separation_r2(const Cloud& c, int64_t i, int64_t j) {
  double d[3];
  for (int k = 0; k < 3; ++k) {
    double dx = c.pos[3 * j + k] - c.pos[3 * i + k];
    if (c.box > 0.0) {
      const double half = 0.5 * c.box;
      if (dx > half) dx = dx - c.box;
      else if (dx < -half) dx = dx + c.box;
    }
    d[k] = dx;
  }
  return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

// k-d tree over all particles: bounding boxes per node, leaves of <= 16.
struct KdNode {
  double lo[3], hi[3];
  int64_t begin, end;   // range in `order`
  int64_t left, right;  // children (-1 for a leaf)
};

struct KdTree {
  std::vector<KdNode> nodes;
  std::vector<int64_t> order;
  double slack;         // absolute slack for pruning (covers rounding)

  void build(const Cloud& c) {
    order.resize(c.n);
    for (int64_t i = 0; i < c.n; ++i) order[i] = i;
    nodes.clear();
    nodes.reserve(2 * (c.n / 8 + 1));
    double amax = c.box;
    for (int64_t i = 0; i < 3 * c.n; ++i) amax = std::max(amax, std::fabs(c.pos[i]));
    slack = 64.0 * std::numeric_limits<double>::epsilon() * (amax + 1e-300);
    if (c.n > 0) build_node(c, 0, c.n);
  }

  int64_t build_node(const Cloud& c, int64_t b, int64_t e) {
    KdNode nd;
    for (int k = 0; k < 3; ++k) { nd.lo[k] = INFINITY; nd.hi[k] = -INFINITY; }
    for (int64_t t = b; t < e; ++t)
      for (int k = 0; k < 3; ++k) {
        const double x = c.pos[3 * order[t] + k];
        nd.lo[k] = std::min(nd.lo[k], x);
        nd.hi[k] = std::max(nd.hi[k], x);
      }
    nd.begin = b; nd.end = e; nd.left = nd.right = -1;
    const int64_t id = (int64_t)nodes.size();
    nodes.push_back(nd);
    if (e - b > 16) {
      int ax = 0;
      for (int k = 1; k < 3; ++k)
        if (nd.hi[k] - nd.lo[k] > nd.hi[ax] - nd.lo[ax]) ax = k;
      const int64_t mid = b + (e - b) / 2;
      std::nth_element(order.begin() + b, order.begin() + mid, order.begin() + e,
                       [&](int64_t p, int64_t q) { return c.pos[3 * p + ax] < c.pos[3 * q + ax]; });
      const int64_t l = build_node(c, b, mid);
      const int64_t r = build_node(c, mid, e);
      nodes[id].left = l; nodes[id].right = r;
    }
    return id;
  }

  // Lower bound of the distance from point p to the node box (periodic aware),
  // minus the rounding slack; never larger than the separation computed by
  // separation_r2 for any particle in the box.
  double box_distance(const Cloud& c, const KdNode& nd, const double* p) const {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
      double best = std::max(std::max(nd.lo[k] - p[k], 0.0), p[k] - nd.hi[k]);
      if (c.box > 0.0) {
        for (int sh = -1; sh <= 1; sh += 2) {
          const double q = p[k] + sh * c.box;
          const double d = std::max(std::max(nd.lo[k] - q, 0.0), q - nd.hi[k]);
          best = std::min(best, d);
        }
      }
      best = std::max(best - slack, 0.0);
      s += best * best;
    }
    return s;
  }

  // Calls f(j, r2) for every j != i with r2 < h*h; f returns false to stop
  // the walk early.  Nearer children are visited first.
  template <class F>
  void for_each_within(const Cloud& c, int64_t i, double h, F&& f) const {
    const double hh = h * h;
    const double* p = c.pos + 3 * i;
    std::vector<int64_t> stack;
    stack.push_back(0);
    while (!stack.empty()) {
      const KdNode& nd = nodes[stack.back()];
      stack.pop_back();
      if (box_distance(c, nd, p) > hh) continue;
      if (nd.left < 0) {
        for (int64_t t = nd.begin; t < nd.end; ++t) {
          const int64_t j = order[t];
          if (j == i) continue;
          const double r2 = separation_r2(c, i, j);
          if (r2 < hh && !f(j, r2)) return;
        }
      } else {
        const double dl = box_distance(c, nodes[nd.left], p);
        const double dr = box_distance(c, nodes[nd.right], p);
        if (dl <= dr) { stack.push_back(nd.right); stack.push_back(nd.left); }
        else { stack.push_back(nd.left); stack.push_back(nd.right); }
      }
    }
  }
};

struct Search {
  const Cloud& c;
  const KdTree* tree;   // null: brute force
  // f(j, r2) returns false to stop early
  template <class F>
  void within_until(int64_t i, double h, F&& f) const {
    if (tree) { tree->for_each_within(c, i, h, f); return; }
    const double hh = h * h;
    for (int64_t j = 0; j < c.n; ++j) {
      if (j == i) continue;
      const double r2 = separation_r2(c, i, j);
      if (r2 < hh && !f(j, r2)) return;
    }
  }
  template <class F>
  void within(int64_t i, double h, F&& f) const {
    within_until(i, h, [&](int64_t j, double r2) { f(j, r2); return true; });
  }
  int64_t count_within(int64_t i, double h) const {
    int64_t k = 0;
    within(i, h, [&](int64_t, double) { ++k; });
    return k;
  }
  // min(c_i(h), cap): the bisection only compares the count with the band,
  // so counting may stop once it exceeds the band.
  int64_t count_capped(int64_t i, double h, int64_t cap) const {
    int64_t k = 0;
    within_until(i, h, [&](int64_t, double) { return ++k < cap; });
    return k;
  }
};

// Starting radius of the bisection, see the header comment.
double initial_h(double l_ext, int64_t n, int n_ngb) {
  int e = 0;
  // largest e with 8^e * n_ngb <= 4 n
  while (e < 60) {
    const double lhs = std::ldexp((double)n_ngb, 3 * (e + 1));
    if (lhs <= 4.0 * (double)n) ++e; else break;
  }
  return std::ldexp(l_ext, -e);
}

// Bisection on the neighbour count; returns h, sets *nonconv on failure.
double bisect_h(const Search& s, int64_t i, double h0, int n_ngb, int tol, int* nonconv,
                int64_t* count_out) {
  double h = h0, lo = 0.0, hi = 0.0;
  bool have_hi = false;
  *nonconv = 1;
  int64_t c = 0;
  for (int it = 0; it < 128; ++it) {
    c = s.count_capped(i, h, (int64_t)n_ngb + tol + 1);
    if (c >= n_ngb - tol && c <= n_ngb + tol) { *nonconv = 0; break; }
    if (c < n_ngb - tol) {
      lo = h;
      h = have_hi ? 0.5 * (lo + hi) : 2.0 * h;
    } else {
      hi = h; have_hi = true;
      h = 0.5 * (lo + hi);
    }
  }
  if (*nonconv) c = s.count_within(i, h);
  *count_out = c;
  return h;
}

const double K8PI = 8.0 / M_PI;           // cubic spline normalisation 8/pi
const double K3_4PI = 3.0 / (4.0 * M_PI); // top-hat normalisation 3/(4 pi)

// W(q) with q = r/h for r < h.  norm = K/((h h) h).
double kernel_norm(int kernel, double h) {
  return (kernel == 1 ? K3_4PI : K8PI) / ((h * h) * h);
}
double kernel_shape(int kernel, double q) {
  if (kernel == 1) return 1.0;
  if (q <= 0.5) return (1.0 - 6.0 * (q * q)) + 6.0 * ((q * q) * q);
  const double u = 1.0 - q;
  return 2.0 * ((u * u) * u);
}

// Tabulated sigma/m(v), Sec. 4.1: linear in log v between nodes, held at
// the end values outside the table.
double sigma_table(const orc_sigma& s, double v) {
  const int n = s.tab_n;
  if (!(v > s.tab_v[0])) return s.tab_s[0];
  if (v >= s.tab_v[n - 1]) return s.tab_s[n - 1];
  int k = 0;
  while (!(v < s.tab_v[k + 1])) ++k;  // v_k <= v < v_{k+1}
  const double t = (std::log(v) - std::log(s.tab_v[k])) /
                   (std::log(s.tab_v[k + 1]) - std::log(s.tab_v[k]));
  return s.tab_s[k] + t * (s.tab_s[k + 1] - s.tab_s[k]);
}

double sigma_over_m(const orc_sigma& s, double vrel) {
  if (s.kind == 2) return sigma_table(s, vrel);
  if (s.kind == 1) {
    const double t = 1.0 + (vrel * vrel) / (s.w * s.w);
    return s.sigma0 / (t * t);
  }
  return s.sigma0;
}

// P(i|j) for j within h_i of i.
double directed_probability(int kernel, const orc_sigma& sig, double m_j, double vrel,
                            double r2, double h_i, double dt_i) {
  const double q = std::sqrt(r2) / h_i;
  const double W = kernel_norm(kernel, h_i) * kernel_shape(kernel, q);
  const double s = sigma_over_m(sig, vrel);
  return ((((0.5 * m_j) * s) * vrel) * W) * dt_i;
}

// ---- kernel-overlap estimator (Eq. 15, Appendix A) ----------------------
// ghat(a, s) = int W(|y|, a) W(|y - s z|, 1 - a) d^3y: the overlap of the
// kernels of two particles a distance s apart, in units of H = h_i + h_j
// (g_ij = ghat / H^3).  Composite Gauss-Legendre in cylindrical coordinates
// (z along the separation) over the lens where both kernels are non-zero.
double overlap_quadrature(int kernel, double a, double s, int panels) {
  const double b = 1.0 - a;
  if (a <= 0.0) return kernel_norm(kernel, 1.0) * kernel_shape(kernel, s < 1.0 ? s : 1.0) *
                       (s < 1.0 ? 1.0 : 0.0);
  if (!(s < a + b)) return 0.0;
  static const double gx[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                               -0.1834346424956498, 0.1834346424956498, 0.5255324099163290,
                               0.7966664774136267, 0.9602898564975363};
  static const double gw[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                               0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                               0.2223810344533745, 0.1012285362903763};
  auto w = [&](double r, double h) {
    const double q = r / h;
    return q < 1.0 ? kernel_norm(kernel, h) * kernel_shape(kernel, q) : 0.0;
  };
  const double z0 = std::max(-a, s - b), z1 = std::min(a, s + b);
  // the lens's radial limit switches from one sphere to the other on the
  // plane where the spheres meet: integrate either side of it separately
  double zc = s > 0.0 ? (a * a - b * b + s * s) / (2.0 * s) : z1;
  if (!(zc > z0 && zc < z1)) zc = z1;
  double total = 0.0;
  for (int pz = 0; pz < 2 * panels; ++pz) {
    const bool first = pz < panels;
    const double lo = first ? z0 : zc, hi = first ? zc : z1;
    if (!(hi > lo)) continue;
    const int k = first ? pz : pz - panels;
    const double za = lo + (hi - lo) * k / panels, zb = lo + (hi - lo) * (k + 1) / panels;
    for (int iz = 0; iz < 8; ++iz) {
      const double z = 0.5 * (za + zb) + 0.5 * (zb - za) * gx[iz];
      const double wz = 0.5 * (zb - za) * gw[iz];
      const double ra2 = a * a - z * z, rb2 = b * b - (z - s) * (z - s);
      if (ra2 <= 0.0 || rb2 <= 0.0) continue;
      const double rmax = std::sqrt(std::min(ra2, rb2));
      double inner = 0.0;
      for (int pr = 0; pr < panels; ++pr) {
        const double ra = rmax * pr / panels, rb = rmax * (pr + 1) / panels;
        for (int ir = 0; ir < 8; ++ir) {
          const double rho = 0.5 * (ra + rb) + 0.5 * (rb - ra) * gx[ir];
          const double wr = 0.5 * (rb - ra) * gw[ir];
          inner += wr * 2.0 * M_PI * rho * w(std::sqrt(rho * rho + z * z), a) *
                   w(std::sqrt(rho * rho + (z - s) * (z - s)), b);
        }
      }
      total += wz * inner;
    }
  }
  return total;
}

// Bilinear interpolation of the table (a in [0, 1/2], s in [0, 1)).
double overlap_hat(const double* T, int na, int ns, double a, double s) {
  if (!(s < 1.0)) return 0.0;
  const double fa = a * (2.0 * (double)na);
  int ia = (int)fa;
  if (ia > na - 1) ia = na - 1;
  const double ta = fa - (double)ia;
  const double fs = s * (double)ns;
  int is = (int)fs;
  if (is > ns - 1) is = ns - 1;
  const double ts = fs - (double)is;
  const double* r0 = T + (int64_t)ia * (ns + 1);
  const double* r1 = r0 + (ns + 1);
  const double g0 = (1.0 - ts) * r0[is] + ts * r0[is + 1];
  const double g1 = (1.0 - ts) * r1[is] + ts * r1[is + 1];
  return (1.0 - ta) * g0 + ta * g1;
}

// g_ij = ghat(min(h_i, h_j) / H, r_ij / H) / H^3, H = h_i + h_j (symmetric in i, j)
double overlap_g(const orc_config& cfg, double hi, double hj, double r2) {
  const double H = hi + hj;
  const double a = std::min(hi, hj) / H;
  const double s = std::sqrt(r2) / H;
  return overlap_hat(cfg.ov_table, cfg.ov_na, cfg.ov_ns, a, s) / ((H * H) * H);
}

// P(i|j) with the overlap factor in place of W(r_ij, h_i)
double overlap_probability(const orc_sigma& sig, double m_j, double vrel, double g,
                           double dt_i) {
  const double s = sigma_over_m(sig, vrel);
  return ((((0.5 * m_j) * s) * vrel) * g) * dt_i;
}

double rel_speed(const double* vi, const double* vj) {
  const double dx = vi[0] - vj[0], dy = vi[1] - vj[1], dz = vi[2] - vj[2];
  return std::sqrt((dx * dx + dy * dy) + dz * dz);
}

// Marsaglia (1972): x1, x2 uniform in (-1, 1), s = x1^2 + x2^2 < 1,
// e = (2 x1 sqrt(1-s), 2 x2 sqrt(1-s), 1 - 2 s).
int isotropic_direction(uint64_t seed, uint64_t step, uint32_t a, uint32_t b, double e[3]) {
  for (uint32_t t = 0; t < 64; ++t) {
    uint32_t w[4];
    draw_words(seed, step, 1u + t, a, b, w);
    const double x1 = 2.0 * uniform53(w[0], w[1]) - 1.0;
    const double x2 = 2.0 * uniform53(w[2], w[3]) - 1.0;
    const double s = x1 * x1 + x2 * x2;
    if (s > 0.0 && s < 1.0) {
      const double k = 2.0 * std::sqrt(1.0 - s);
      e[0] = x1 * k; e[1] = x2 * k; e[2] = 1.0 - 2.0 * s;
      return 1;
    }
  }
  e[0] = 0.0; e[1] = 0.0; e[2] = 1.0;
  return 0;
}

// Kick in the centre-of-momentum frame (Sec. 4.1): the pair keeps its
// centre-of-momentum velocity and leaves along +-e with relative speed
// eps |v_i - v_j| (eps = 1: elastic).
void kick(double mi, double mj, double* vi, double* vj, const double e[3], double eps) {
  const double M = mi + mj;
  double vc[3];
  for (int k = 0; k < 3; ++k) vc[k] = ((mi * vi[k]) + (mj * vj[k])) / M;
  const double g = rel_speed(vi, vj) * eps;
  const double fi = (mj * g) / M, fj = (mi * g) / M;
  for (int k = 0; k < 3; ++k) {
    vi[k] = vc[k] + fi * e[k];
    vj[k] = vc[k] - fj * e[k];
  }
}

// Neumaier-compensated sum.
struct CSum {
  double s = 0.0, c = 0.0;
  void add(double x) {
    const double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

void conserved(int64_t n, const double* mass, const double* vel, double* e, double p[3]) {
  CSum se, sp[3];
  for (int64_t i = 0; i < n; ++i) {
    const double* v = vel + 3 * i;
    const double v2 = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
    se.add(0.5 * mass[i] * v2);
    for (int k = 0; k < 3; ++k) sp[k].add(mass[i] * v[k]);
  }
  *e = se.value();
  for (int k = 0; k < 3; ++k) p[k] = sp[k].value();
}

struct Pair {
  uint64_t ord;
  uint32_t a, b;      // ids, a < b
  int64_t i, j;       // storage indices of the a- and b-particle
  double p;           // P_pair
};

// Canonical application of the accepted pairs (Sec. 4.1 kick; Sec. 4.4:
// a particle may scatter several times in one step, each kick seeing the
// velocities the earlier ones left).  The pairs are put in ascending
// (ord, a, b) order -- a stable sort, so records with equal keys keep the
// order they were given in -- and kicked one after another.  Returns the
// number of direction draws that ran out of tries.
int64_t apply_pairs(std::vector<Pair>& acc, double* vel, const double* mass, uint64_t seed,
                    uint64_t step, double eps) {
  std::stable_sort(acc.begin(), acc.end(), [](const Pair& x, const Pair& y) {
    if (x.ord != y.ord) return x.ord < y.ord;
    if (x.a != y.a) return x.a < y.a;
    return x.b < y.b;
  });
  int64_t dir_fail = 0;
  for (const Pair& pr : acc) {
    double e[3];
    if (!isotropic_direction(seed, step, pr.a, pr.b, e)) ++dir_fail;
    kick(mass[pr.i], mass[pr.j], vel + 3 * pr.i, vel + 3 * pr.j, e, eps);
  }
  return dir_fail;
}

}  // namespace

extern "C" {

void orc_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4]) {
  philox4x32_10(key, ctr, out);
}

double orc_uniform53(uint32_t wa, uint32_t wb) { return uniform53(wa, wb); }

double orc_kernel_w(int kernel, double r, double h) {
  if (!(r < h)) return 0.0;
  return kernel_norm(kernel, h) * kernel_shape(kernel, r / h);
}

double orc_sigma_over_m(const orc_sigma* s, double vrel) { return sigma_over_m(*s, vrel); }

double orc_overlap_quadrature(int kernel, double a, double s, int panels) {
  return overlap_quadrature(kernel, a, s, panels);
}

// The table of the overlap estimator: ghat(k / (2 na), l / ns), row-major in a.
void orc_overlap_table(int kernel, int na, int ns, int panels, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k <= na; ++k)
    for (int l = 0; l <= ns; ++l)
      out[(int64_t)k * (ns + 1) + l] =
          overlap_quadrature(kernel, 0.5 * (double)k / (double)na, (double)l / (double)ns, panels);
}

double orc_overlap_g(const orc_config* cfg, double hi, double hj, double r2) {
  return overlap_g(*cfg, hi, hj, r2);
}

double orc_directed_probability(int kernel, const orc_sigma* sig, double m_j,
                                const double* vi, const double* vj, double r2,
                                double h_i, double dt_i) {
  return directed_probability(kernel, *sig, m_j, rel_speed(vi, vj), r2, h_i, dt_i);
}

int orc_direction(uint64_t seed, uint64_t step, uint32_t a, uint32_t b, double e[3]) {
  return isotropic_direction(seed, step, a, b, e);
}

void orc_kick(double mi, double mj, double* vi, double* vj, const double e[3], double eps) {
  kick(mi, mj, vi, vj, e, eps);
}

double orc_initial_h(double l_ext, int64_t n, int n_ngb) { return initial_h(l_ext, n, n_ngb); }

// Neighbour counts c_i(h) for a list of query particles (brute force or tree).
void orc_counts(int64_t n, const double* pos, double box, int use_tree, int64_t nq,
                const int64_t* q, const double* h, int64_t* out) {
  Cloud c{n, pos, box};
  KdTree tree;
  if (use_tree) tree.build(c);
  Search s{c, use_tree ? &tree : nullptr};
  for (int64_t t = 0; t < nq; ++t) out[t] = s.count_within(q[t], h[t]);
}

// h_SI of a list of query particles (used to sample large workloads).
void orc_h_for(const orc_config* cfg, int64_t n, const double* pos, int64_t nq,
               const int64_t* q, double* h_out, int64_t* count_out, int* nonconv_out) {
  Cloud c{n, pos, cfg->box};
  KdTree tree;
  if (cfg->use_tree) tree.build(c);
  Search s{c, cfg->use_tree ? &tree : nullptr};
  double l_ext = cfg->box;
  if (!(l_ext > 0.0)) {
    l_ext = 0.0;
    for (int k = 0; k < 3; ++k) {
      double lo = INFINITY, hi = -INFINITY;
      for (int64_t i = 0; i < n; ++i) { lo = std::min(lo, pos[3 * i + k]); hi = std::max(hi, pos[3 * i + k]); }
      l_ext = std::max(l_ext, hi - lo);
    }
  }
  const double h0 = initial_h(l_ext, n, cfg->n_ngb);
#pragma omp parallel for schedule(dynamic, 64) num_threads(cfg->n_threads > 0 ? cfg->n_threads : omp_get_max_threads())
  for (int64_t t = 0; t < nq; ++t) {
    int nc = 0; int64_t cnt = 0;
    h_out[t] = bisect_h(s, q[t], h0, cfg->n_ngb, cfg->ngb_tol, &nc, &cnt);
    if (count_out) count_out[t] = cnt;
    if (nonconv_out) nonconv_out[t] = nc;
  }
}

// Step 7 alone: applies n_pairs given accepted pairs (ord, ids a < b,
// storage indices ia, ib) to vel (n x 3, in place) in the canonical order,
// elastic when eps = 1.  Returns the number of exhausted direction draws,
// or -1 if an index lies outside [0, n) or names one particle twice.
int64_t orc_apply_pairs(int64_t n, int64_t n_pairs, const uint64_t* ord, const uint32_t* a,
                        const uint32_t* b, const int64_t* ia, const int64_t* ib, double* vel,
                        const double* mass, uint64_t seed, uint64_t step, double eps) {
  std::vector<Pair> acc((size_t)n_pairs);
  for (int64_t k = 0; k < n_pairs; ++k) {
    if (ia[k] < 0 || ia[k] >= n || ib[k] < 0 || ib[k] >= n || ia[k] == ib[k]) return -1;
    acc[k] = Pair{ord[k], a[k], b[k], ia[k], ib[k], 0.0};
  }
  return apply_pairs(acc, vel, mass, seed, step, eps);
}

// One scattering step.  pos/vel are n x 3 row-major; vel is updated in place.
// h_out / dtlim_out are written for active particles only.  Accepted pairs
// (sorted by (ord, a, b)) go to pair_ab[2k], pair_ab[2k+1], pair_ord[k],
// pair_p[k] for k < min(count, max_pairs); *n_pairs_out receives the count.
// Returns 0, or -1 on invalid arguments.
int orc_step(const orc_config* cfg, int64_t n, const double* pos, double* vel,
             const double* mass, const uint32_t* ids, const uint8_t* active,
             const int8_t* bins, double dt_max, const orc_sigma* sig, uint64_t seed,
             uint64_t step, double* h_out, double* dtlim_out, int64_t max_pairs,
             uint32_t* pair_ab, uint64_t* pair_ord, double* pair_p, int64_t* n_pairs_out,
             orc_stats* st) {
  if (n < 0 || !cfg || !sig) return -1;
  const int nthr = cfg->n_threads > 0 ? cfg->n_threads : omp_get_max_threads();
  Cloud c{n, pos, cfg->box};
  KdTree tree;
  if (cfg->use_tree && n > 0) tree.build(c);
  Search s{c, cfg->use_tree ? &tree : nullptr};

  orc_stats S;
  std::memset(&S, 0, sizeof(S));
  conserved(n, mass, vel, &S.e_before, S.p_before);

  std::vector<int64_t> act;
  for (int64_t i = 0; i < n; ++i)
    if (!active || active[i]) act.push_back(i);
  S.n_active = (int64_t)act.size();

  // extent for the starting radius
  double l_ext = cfg->box;
  if (!(l_ext > 0.0)) {
    l_ext = 0.0;
    for (int k = 0; k < 3; ++k) {
      double lo = INFINITY, hi = -INFINITY;
      for (int64_t i = 0; i < n; ++i) { lo = std::min(lo, pos[3 * i + k]); hi = std::max(hi, pos[3 * i + k]); }
      if (n > 0) l_ext = std::max(l_ext, hi - lo);
    }
  }
  const double h0 = initial_h(l_ext, n, cfg->n_ngb);

  // 1. smoothing lengths of the active particles (of every particle for the
  // overlap estimator, whose neighbours are those with r_ij < h_i + h_j)
  const bool overlap = cfg->estimator == 1;
  std::vector<double> h(n, 0.0);
  std::vector<char> is_act(n, 0);
  for (int64_t i : act) is_act[i] = 1;
  std::vector<int64_t> all;
  if (overlap)
    for (int64_t i = 0; i < n; ++i) all.push_back(i);
  const std::vector<int64_t>& hset = overlap ? all : act;
  int64_t nonconv = 0;
#pragma omp parallel for schedule(dynamic, 32) num_threads(nthr) reduction(+ : nonconv)
  for (int64_t t = 0; t < (int64_t)hset.size(); ++t) {
    const int64_t i = hset[t];
    if (cfg->fixed_h > 0.0) { h[i] = cfg->fixed_h; continue; }
    int nc = 0; int64_t cnt = 0;
    h[i] = bisect_h(s, i, h0, cfg->n_ngb, cfg->ngb_tol, &nc, &cnt);
    nonconv += nc;
  }
  S.n_h_nonconv = nonconv;

  auto dt_of = [&](int64_t i) { return std::ldexp(dt_max, -(int)bins[i]); };
  double h_max = 0.0;
  if (overlap)
    for (int64_t i = 0; i < n; ++i) h_max = std::max(h_max, h[i]);

  // 2. candidate pairs, drawn once each, and (v sigma/m)_max per active particle
  std::vector<std::vector<Pair>> acc_t(nthr);
  std::vector<double> vsmax(n, 0.0);
  int64_t n_cand = 0, n_pge1 = 0;
  std::vector<double> psum(n, 0.0);
#pragma omp parallel for schedule(dynamic, 32) num_threads(nthr) reduction(+ : n_cand, n_pge1)
  for (int64_t t = 0; t < (int64_t)act.size(); ++t) {
    const int64_t i = act[t];
    const int tid = omp_get_thread_num();
    double vs = 0.0;
    s.within(i, overlap ? h[i] + h_max : h[i], [&](int64_t j, double r2) {
      if (overlap) {
        const double H = h[i] + h[j];
        if (!(r2 < H * H)) return;               // not overlapping
      }
      const double vrel = rel_speed(vel + 3 * i, vel + 3 * j);
      vs = std::max(vs, vrel * sigma_over_m(*sig, vrel));
      // j sees i: j active and i in its neighbour set (symmetric for the overlap)
      const bool j_sees_i = is_act[j] && (overlap || r2 < h[j] * h[j]);
      if (j_sees_i && ids[j] < ids[i]) return;   // j owns the pair
      ++n_cand;
      double p_i, p_j = 0.0;
      if (overlap) {
        const double g = overlap_g(*cfg, h[i], h[j], r2);
        p_i = overlap_probability(*sig, mass[j], vrel, g, dt_of(i));
        if (j_sees_i) p_j = overlap_probability(*sig, mass[i], vrel, g, dt_of(j));
      } else {
        p_i = directed_probability(cfg->kernel, *sig, mass[j], vrel, r2, h[i], dt_of(i));
        if (j_sees_i) p_j = directed_probability(cfg->kernel, *sig, mass[i], vrel, r2, h[j], dt_of(j));
      }
      const bool i_is_a = ids[i] < ids[j];
      const double p_pair = i_is_a ? (p_i + p_j) : (p_j + p_i);
      if (p_pair >= 1.0) ++n_pge1;
      psum[i] += p_pair;
      const uint32_t a = i_is_a ? ids[i] : ids[j], b = i_is_a ? ids[j] : ids[i];
      uint32_t w[4];
      draw_words(seed, step, 0u, a, b, w);
      const double u = uniform53(w[0], w[1]);
      if (u < p_pair) {
        Pair pr;
        pr.ord = ((uint64_t)w[2] << 32) | (uint64_t)w[3];
        pr.a = a; pr.b = b;
        pr.i = i_is_a ? i : j; pr.j = i_is_a ? j : i;
        pr.p = p_pair;
        acc_t[tid].push_back(pr);
      }
    });
    vsmax[i] = vs;
  }
  S.n_candidate_pairs = n_cand;
  S.n_p_ge_1 = n_pge1;
  {
    CSum sp;
    for (int64_t i : act) sp.add(psum[i]);
    S.sum_p = sp.value();
  }

  // 3. canonical order and sequential application with current velocities
  std::vector<Pair> acc;
  for (auto& v : acc_t) acc.insert(acc.end(), v.begin(), v.end());
  S.n_accepted = (int64_t)acc.size();
  S.n_dir_fail = apply_pairs(acc, vel, mass, seed, step, 1.0 - sig->inelastic);

  // 4. outputs for the active particles: h and the Eq. 18 limit (h of every
  // particle for the overlap estimator)
  if (overlap && h_out)
    for (int64_t i = 0; i < n; ++i) h_out[i] = h[i];
  for (int64_t i : act) {
    if (h_out) h_out[i] = h[i];
    if (dtlim_out) {
      const double den = (mass[i] * kernel_norm(cfg->kernel, h[i])) * vsmax[i];
      dtlim_out[i] = vsmax[i] > 0.0 ? (cfg->c_sidm * 2.0) / den : INFINITY;
    }
  }
  for (int64_t k = 0; k < (int64_t)acc.size() && k < max_pairs; ++k) {
    if (pair_ab) { pair_ab[2 * k] = acc[k].a; pair_ab[2 * k + 1] = acc[k].b; }
    if (pair_ord) pair_ord[k] = acc[k].ord;
    if (pair_p) pair_p[k] = acc[k].p;
  }
  if (n_pairs_out) *n_pairs_out = (int64_t)acc.size();
  conserved(n, mass, vel, &S.e_after, S.p_after);
  if (st) *st = S;
  return 0;
}

}  // extern "C"
