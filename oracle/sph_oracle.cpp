/*
 * sph_oracle.cpp -- plain FP64 CPU oracle for the SPH density / gradient /
 * force pair loops and the Newton iteration on the smoothing length, written
 * from the equations of "Task-parallelism in SWIFT for heterogeneous compute
 * architectures" (arXiv 2505.14538), Sec. 2.1.
 *
 * TEST INFRASTRUCTURE. This library exists to check the CUDA path. Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it. It shares no code, header, table or constant with the CUDA path.
 *
 * Everything here is the plain definition: for every particle i, loop over
 * every candidate j (all particles, or the 27 cells around i when a cell list
 * is requested), apply the neighbour predicate, and accumulate the sums the
 * paper writes down, in double precision, in j order. No blocking, no fusion.
 *
 * Readings of the paper taken here (the paper is silent or garbled on each):
 *  - Kernel: cubic spline (M4) in 3D with compact support H = kernel_gamma*h
 *    (Sec. 2.1.3, "H_i = gamma_k h_i"); W = (8/pi) H^-3 w(r/H),
 *    w(q) = 1-6q^2+6q^3 (q<1/2), 2(1-q)^3 (1/2<=q<1), 0 beyond.
 *    Sec. 2.1.1 also names the Wendland kernels; with kernel = 1 or 2:
 *    Wendland C2, W = (21/(2 pi)) H^-3 (1-q)^4 (1+4q), and Wendland C4,
 *    W = (495/(32 pi)) H^-3 (1-q)^6 (1+6q+35q^2/3) (the 3-D normalisations;
 *    their own H/h from the same second-moment definition as the cubic
 *    spline's, sqrt(15)/2 and sqrt(78)/4, is passed as kernel_gamma).
 *  - Eq. 6: "grad_i W_ij" is the scalar dW/dr (it is multiplied by r_ij/h_i).
 *  - Eq. 3/4: differenced form. div v_i = (1/rho_i) sum_j m_j (v_j-v_i).grad_i W_ij;
 *    curl v_i = (1/rho_i) sum_j m_j (v_i-v_j) x grad_i W_ij. Eq. 4 as printed
 *    has the opposite sign to Eq. 3 under either gradient convention; the sign
 *    taken here returns +2*Omega for a rigid rotation v = Omega x r.
 *  - h iteration (Sec. 2.1.2): Newton on F(h) = n(h) - (eta/h)^3 with
 *    F'(h) = dn/dh + 3 eta^3/h^4; step clamped to [h/2, 2h]; bisection on a
 *    maintained bracket when F' <= 0 or the step leaves the bracket; converged
 *    when |F| <= h_tol (eta/h)^3; capped at h_max (not converged when the cap
 *    binds); outputs always belong to the last h at which the sums were taken.
 *  - Eq. 8: Omega_i = 1 + h_i/(3 rho_i) drho_i/dh, and the force loop multiplies
 *    by f_i = 1/Omega_i (grad-h correction).
 *  - Ghost: P = (gamma-1) rho u, c = sqrt(gamma (gamma-1) u), Balsara switch
 *    B = |div v| / (|div v| + |curl v| + 1e-4 c/h), B = 0 when div v = 0.
 *  - Gradient loop: v_sig,max over j in N_i and i itself of c_i+c_j-beta mu_ij
 *    (Eq. 10-11) and the Brookshaw Laplacian
 *    lap u_i = 2 sum_j (m_j/rho_j)(u_i-u_j) (dW/dr)(r,h_i)/r.
 *  - Force loop, pair set r < max(H_i, H_j):
 *      Eq. 17 with the second f_i read as f_j and the j term taken at h_j;
 *      Eq. 18 at h_i;
 *      Eq. 7/9: nu_ij = -alpha_v,ij mu_ij v_sig,ij / (rho_i+rho_j) >= 0
 *        (Eq. 9 as printed is dimensionally inconsistent), acceleration
 *        -m_j nu_ij (f_i G_i + f_j G_j)/2 and the matching heating term
 *        +m_j nu_ij v_ij.(f_i G_i + f_j G_j)/4 so energy is conserved;
 *      Eq. 16 alpha_v,ij with per-particle alpha_v and B;
 *      Eq. 19, 20, 22: conduction with v_c = |v_ij.r_hat| + sqrt(2|P_i-P_j|/(rho_i+rho_j))
 *        and kernel factor (f_i dW_i + f_j dW_j), symmetric in i,j;
 *      dh/dt = -(h_i/(3 rho_i)) f_i sum_j m_j v_ij.G_i (grad-h continuity).
 *  - Neighbour predicate, in FP64 from the given coordinates:
 *      dx = x_i - x_j, dx -= L*round(dx/L) when periodic, r2 = (dx^2+dy^2)+dz^2,
 *      H = kernel_gamma*h, density/gradient: j != i and r2 < H_i*H_i (self added
 *      separately), force: r2 < H_i*H_i or r2 < H_j*H_j.
 *  - Cell id: wrap x into [0,L) in FP64, cell = floor(x*nc/L) clamped to nc-1,
 *    linear id = cx + nc*(cy + nc*cz).
 *
 * Pins (tests/test_oracle_*.py) tie these to values the paper or the
 * mathematics fixes. The paper prints no worked example of the force terms,
 * so their magnitudes are pinned to continuum limits: the pressure term to
 * -(1/rho) dp/dr of the Gresho-Chan profile (Eq. 28), the viscosity (the
 * Eq. 9 reading above) to its heating under homologous compression, the
 * conduction (Eqs. 19, 20, 22) to its value at the minimum of a quadratic u,
 * each in closed form in the kernel's radial moments.
 *
 * Build: g++ -O2 -std=c++17 -fopenmp -fPIC -shared -ffp-contract=off
 * (no FMA contraction, so every operation rounds exactly as written).
 */
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
  double box[3];
  int periodic;
  double gamma_eos;     /* adiabatic index */
  double eta;           /* resolution eta: target n = (eta/h)^3 */
  double kernel_gamma;  /* H/h */
  double alpha_v;       /* viscosity alpha (used when no per-particle array) */
  double beta_v;        /* signal-velocity beta (Eq. 10) */
  double alpha_c;       /* conduction alpha (used when no per-particle array) */
  double h_tol;         /* Newton tolerance on |F|/(eta/h)^3 */
  int max_iter;
  double h_max;         /* cap on h; <= 0 means none */
  int use_cells;        /* 0: all pairs (brute force); 1: cell list */
  int nthreads;         /* <= 0: OpenMP default */
  int terms;            /* force-loop terms: 1 pressure/energy, 2 viscosity, 4 conduction */
  int kernel;           /* 0 cubic spline, 1 Wendland C2, 2 Wendland C4 */
} oracle_params;

}  // extern "C"

namespace {

/* ------------------------------------------------------------------ */
/* Op-counting scalar: the pair functions below are templates so the   */
/* same code that computes the oracle's values also counts its flops   */
/* (add/sub/mul = 1, div = 1, sqrt = 1, comparisons counted apart).    */
/* ------------------------------------------------------------------ */
struct OpTally {
  long long add, mul, div, sqrt, cmp;
};
thread_local OpTally* g_tally = nullptr;

struct Cnt {
  double v;
  Cnt(double x = 0.0) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { if (g_tally) g_tally->add++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { if (g_tally) g_tally->add++; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { if (g_tally) g_tally->mul++; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { if (g_tally) g_tally->div++; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline bool operator<(Cnt a, Cnt b) { if (g_tally) g_tally->cmp++; return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { if (g_tally) g_tally->cmp++; return a.v > b.v; }
inline double val(Cnt a) { return a.v; }
inline double val(double a) { return a; }
inline Cnt sqrt_(Cnt a) { if (g_tally) g_tally->sqrt++; return Cnt(std::sqrt(a.v)); }
inline double sqrt_(double a) { return std::sqrt(a); }
inline Cnt abs_(Cnt a) { return Cnt(std::fabs(a.v)); }
inline double abs_(double a) { return std::fabs(a); }
inline Cnt min0_(Cnt a) { if (g_tally) g_tally->cmp++; return Cnt(a.v < 0.0 ? a.v : 0.0); }
inline double min0_(double a) { return a < 0.0 ? a : 0.0; }
inline Cnt max_(Cnt a, Cnt b) { if (g_tally) g_tally->cmp++; return Cnt(a.v > b.v ? a.v : b.v); }
inline double max_(double a, double b) { return a > b ? a : b; }

const double kPi = 3.14159265358979323846;

/* Cubic spline (M4) shape w(q) and dw/dq on the support q in [0,1). */
template <class T>
inline void spline(T q, T& w, T& dw) {
  if (q < T(0.5)) {
    w = T(1.0) - T(6.0) * q * q + T(6.0) * q * q * q;
    dw = T(-12.0) * q + T(18.0) * q * q;
  } else if (q < T(1.0)) {
    T s = T(1.0) - q;
    w = T(2.0) * s * s * s;
    dw = T(-6.0) * s * s;
  } else {
    w = T(0.0);
    dw = T(0.0);
  }
}

/* Wendland C2 and C4 shapes w(q) and dw/dq on q in [0,1), zero beyond. */
template <class T>
inline void wendland(int kind, T q, T& w, T& dw) {
  if (!(q < T(1.0))) {
    w = T(0.0);
    dw = T(0.0);
    return;
  }
  T s = T(1.0) - q;
  T s2 = s * s;
  if (kind == 1) {
    w = s2 * s2 * (T(1.0) + T(4.0) * q);
    dw = T(-20.0) * q * s2 * s;
  } else {
    w = s2 * s2 * s2 * (T(1.0) + T(6.0) * q + T(35.0 / 3.0) * q * q);
    dw = T(-56.0 / 3.0) * q * (T(1.0) + T(5.0) * q) * s2 * s2 * s;
  }
}

/* 3-D normalisation C of W = C H^-3 w(r/H) (the integral of W is 1). */
inline double kernel_norm(int kind) {
  return kind == 1 ? 21.0 / (2.0 * kPi) : kind == 2 ? 495.0 / (32.0 * kPi) : 8.0 / kPi;
}

/* Per-particle kernel constants for support H: W = c3 w(q), dW/dr = c4 w'(q). */
template <class T>
struct KernelI {
  T H, invH, c3, c4;
  int kind;
};
template <class T>
inline KernelI<T> kernel_consts(double h, double kernel_gamma, int kind) {
  KernelI<T> k;
  double H = kernel_gamma * h;
  k.H = T(H);
  k.invH = T(1.0 / H);
  k.c3 = T(kernel_norm(kind) / (H * H * H));
  k.c4 = T(kernel_norm(kind) / (H * H * H * H));
  k.kind = kind;
  return k;
}

/* W(r,h) and dW/dr(r,h). */
template <class T>
inline void kernel_eval(const KernelI<T>& k, T r, T& W, T& dWdr) {
  T w, dw;
  if (k.kind == 0) spline(r * k.invH, w, dw);
  else wendland(k.kind, r * k.invH, w, dw);
  W = k.c3 * w;
  dWdr = k.c4 * dw;
}

/* ---------------------------- geometry ----------------------------- */
struct Geo {
  double L[3];
  int periodic;
};

inline void min_image(const Geo& g, double d[3]) {
  if (!g.periodic) return;
  for (int a = 0; a < 3; ++a) d[a] = d[a] - g.L[a] * std::round(d[a] / g.L[a]);
}

inline double r2_of(const double d[3]) { return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]; }

/* Candidate enumeration: brute force or a cell list of width >= rmax. */
struct Cells {
  int nc[3] = {0, 0, 0};
  bool on = false;
  std::vector<std::vector<int64_t>> members;
  std::vector<int> cell_of;
};

inline int cell_coord(double x, double L, int nc) {
  double xw = x - L * std::floor(x / L);
  int c = (int)std::floor(xw * nc / L);
  if (c < 0) c = 0;
  if (c > nc - 1) c = nc - 1;
  return c;
}

Cells make_cells(const Geo& g, int64_t n, const double* x, double rmax, int want) {
  Cells c;
  if (!want || !g.periodic) return c;
  for (int a = 0; a < 3; ++a) {
    c.nc[a] = (int)std::floor(g.L[a] / rmax);
    if (c.nc[a] < 3) return c; /* 27 distinct neighbour cells need >= 3 per axis */
    if (c.nc[a] > 256) c.nc[a] = 256;
  }
  c.on = true;
  c.members.resize((size_t)c.nc[0] * c.nc[1] * c.nc[2]);
  c.cell_of.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    int cx = cell_coord(x[3 * i + 0], g.L[0], c.nc[0]);
    int cy = cell_coord(x[3 * i + 1], g.L[1], c.nc[1]);
    int cz = cell_coord(x[3 * i + 2], g.L[2], c.nc[2]);
    int id = cx + c.nc[0] * (cy + c.nc[1] * cz);
    c.cell_of[i] = id;
    c.members[id].push_back(i);
  }
  return c;
}

/* Calls fn(j) for every candidate j of particle i (including i itself). */
template <class Fn>
inline void for_candidates(const Cells& c, int64_t n, int64_t i, Fn fn) {
  if (!c.on) {
    for (int64_t j = 0; j < n; ++j) fn(j);
    return;
  }
  int id = c.cell_of[i];
  int cx = id % c.nc[0], cy = (id / c.nc[0]) % c.nc[1], cz = id / (c.nc[0] * c.nc[1]);
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int ax = (cx + dx + c.nc[0]) % c.nc[0];
        int ay = (cy + dy + c.nc[1]) % c.nc[1];
        int az = (cz + dz + c.nc[2]) % c.nc[2];
        for (int64_t j : c.members[ax + c.nc[0] * (ay + c.nc[1] * az)]) fn(j);
      }
}

/* ------------------------- density loop ---------------------------- */
template <class T>
struct DensAcc {
  T n, dn, rho, drho, div, cx, cy, cz; /* dn, drho hold sum(3W + r dW/dr) */
  long long count;
};

/* One interacting pair (i, j), j may equal i (then d = 0). d = x_i - x_j. */
template <class T>
inline void density_pair(const KernelI<T>& k, T r2, T dx, T dy, T dz, T mj, T dvx, T dvy, T dvz,
                         bool self, DensAcc<T>& a) {
  T r = sqrt_(r2);
  T W, dWdr;
  kernel_eval(k, r, W, dWdr);
  a.n += W;                                   /* Eq. 5 */
  a.rho += mj * W;                            /* Eq. 2 */
  T t = T(3.0) * W + r * dWdr;                /* n_d W + r dW/dr (Eq. 6) */
  a.dn += t;
  a.drho += mj * t;
  if (!self) {
    a.count++;
    T g = dWdr / r;                           /* grad_i W_ij = g (x_i - x_j) */
    /* dv = v_j - v_i */
    a.div += mj * g * (dvx * dx + dvy * dy + dvz * dz);               /* Eq. 3 */
    /* (v_i - v_j) x (g d) = -(dv x d) g */
    a.cx -= mj * g * (dvy * dz - dvz * dy);                           /* Eq. 4 */
    a.cy -= mj * g * (dvz * dx - dvx * dz);
    a.cz -= mj * g * (dvx * dy - dvy * dx);
  }
}

/* The two sums the h iteration needs, Eq. 5 (n) and Eq. 6 (dn/dh), for one pair. */
template <class T>
inline void number_pair(const KernelI<T>& k, T r2, T& n, T& dn) {
  T r = sqrt_(r2);
  T W, dWdr;
  kernel_eval(k, r, W, dWdr);
  n += W;
  dn += T(3.0) * W + r * dWdr;
}

struct DensOut {
  double n, dn_dh, rho, drho_dh, div, curl[3];
  long long count;
};

/* Eq. 5 and Eq. 6 at h (self included in the sums, not in the count). */
DensOut number_at(const Geo& g, const Cells& c, int64_t n, const double* x, int64_t i, double h,
                  double kernel_gamma, int kind) {
  KernelI<double> k = kernel_consts<double>(h, kernel_gamma, kind);
  double H2 = k.H * k.H;
  double s = 0.0, ds = 0.0;
  long long count = 0;
  for_candidates(c, n, i, [&](int64_t j) {
    double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
    min_image(g, d);
    double r2 = r2_of(d);
    bool self = (j == i);
    if (!self && !(r2 < H2)) return;
    number_pair<double>(k, self ? 0.0 : r2, s, ds);
    if (!self) count++;
  });
  DensOut o{};
  o.n = s;
  o.dn_dh = -ds / h;
  o.count = count;
  return o;
}

DensOut density_at(const Geo& g, const Cells& c, int64_t n, const double* x, const double* v,
                   const double* m, int64_t i, double h, double kernel_gamma, int kind) {
  KernelI<double> k = kernel_consts<double>(h, kernel_gamma, kind);
  double H2 = k.H * k.H;
  DensAcc<double> a{0, 0, 0, 0, 0, 0, 0, 0, 0};
  for_candidates(c, n, i, [&](int64_t j) {
    double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
    min_image(g, d);
    double r2 = r2_of(d);
    bool self = (j == i);
    if (!self && !(r2 < H2)) return;
    density_pair<double>(k, self ? 0.0 : r2, d[0], d[1], d[2], m[j], v[3 * j] - v[3 * i],
                         v[3 * j + 1] - v[3 * i + 1], v[3 * j + 2] - v[3 * i + 2], self, a);
  });
  DensOut o;
  o.n = a.n;
  o.dn_dh = -a.dn / h;
  o.rho = a.rho;
  o.drho_dh = -a.drho / h;
  o.div = a.div / a.rho;
  o.curl[0] = a.cx / a.rho;
  o.curl[1] = a.cy / a.rho;
  o.curl[2] = a.cz / a.rho;
  o.count = a.count;
  return o;
}

/* Newton-Raphson on F(h) = n(h) - (eta/h)^3 (Sec. 2.1.2). Each iteration
 * takes Eq. 5 and Eq. 6 at the current h; the remaining density sums are
 * taken once, at the h the iteration ends on. */
struct SolveOut {
  double h;
  int iters;
  int converged;
  long long pairs;  /* neighbour pairs summed over every pass */
  DensOut d;
};

SolveOut solve_h(const Geo& g, const Cells& c, int64_t n, const double* x, const double* v,
                 const double* m, int64_t i, double h0, const oracle_params& p) {
  const double eta3 = p.eta * p.eta * p.eta;
  const double hmax = p.h_max > 0 ? p.h_max : std::numeric_limits<double>::infinity();
  double h = std::min(h0, hmax);
  double lo = 0.0, hi = std::numeric_limits<double>::infinity();
  SolveOut s;
  s.converged = 0;
  s.pairs = 0;
  for (int it = 0; it < p.max_iter; ++it) {
    DensOut d = number_at(g, c, n, x, i, h, p.kernel_gamma, p.kernel);
    s.pairs += d.count;
    double target = eta3 / (h * h * h);
    double F = d.n - target;
    s.h = h;
    s.iters = it + 1;
    if (std::fabs(F) <= p.h_tol * target) {
      s.converged = 1;
      break;
    }
    if (it == p.max_iter - 1) break;
    if (F < 0.0) lo = std::max(lo, h);
    else hi = std::min(hi, h);
    if (F < 0.0 && h >= hmax) break; /* cannot grow past the cap */
    double Fp = d.dn_dh + 3.0 * eta3 / (h * h * h * h);
    double hn = (Fp > 0.0) ? h - F / Fp : std::numeric_limits<double>::quiet_NaN();
    if (hn == hn) hn = std::min(std::max(hn, 0.5 * h), 2.0 * h);
    if (!(hn == hn) || !(hn > lo) || !(hn < hi)) {
      if (std::isfinite(hi) && lo > 0.0) hn = 0.5 * (lo + hi);
      else if (!std::isfinite(hi)) hn = 2.0 * h;
      else hn = 0.5 * h;
    }
    h = std::min(hn, hmax);
  }
  s.d = density_at(g, c, n, x, v, m, i, s.h, p.kernel_gamma, p.kernel);
  return s;
}

/* ------------------------- gradient loop --------------------------- */
template <class T>
struct GradAcc {
  T vsig, lap;
};

template <class T>
inline void gradient_pair(const KernelI<T>& k, T r2, T dx, T dy, T dz, T dvx, T dvy, T dvz, T ci,
                          T cj, T mj, T rhoj, T du, T beta, GradAcc<T>& a) {
  /* d = x_i - x_j, dv = v_i - v_j, du = u_i - u_j */
  T r = sqrt_(r2);
  T W, dWdr;
  kernel_eval(k, r, W, dWdr);
  T mu = min0_((dvx * dx + dvy * dy + dvz * dz) / r);  /* Eq. 11 */
  T vs = ci + cj - beta * mu;                          /* Eq. 10 */
  a.vsig = max_(a.vsig, vs);
  a.lap += mj / rhoj * du * dWdr / r;                  /* Brookshaw Laplacian */
}

/* --------------------------- force loop ---------------------------- */
template <class T>
struct ForceI {
  KernelI<T> k;
  T f, A, rho, P, c, B, av, ac, u;
};
template <class T>
struct ForceAcc {
  T ax, ay, az, du, dh, sa, su;
};

/* One pair of the force loop; d = x_i - x_j, dv = v_i - v_j. */
template <class T>
inline void force_pair(const ForceI<T>& I, const ForceI<T>& J, T r2, T dx, T dy, T dz, T dvx, T dvy,
                       T dvz, T mj, T beta, int terms, bool scales, ForceAcc<T>& a) {
  T r = sqrt_(r2);
  T invr = T(1.0) / r;
  T ex = dx * invr, ey = dy * invr, ez = dz * invr; /* r_hat */
  T Wi, dWi, Wj, dWj;
  kernel_eval(I.k, r, Wi, dWi); /* zero beyond H_i */
  kernel_eval(J.k, r, Wj, dWj); /* zero beyond H_j */
  T vr = dvx * ex + dvy * ey + dvz * ez;
  T fsum = I.f * dWi + J.f * dWj;
  T acc_s = T(0.0); /* scalar multiplying -r_hat in a_i */
  if (terms & 1) {
    T ps = mj * (I.A * dWi + J.A * dWj);     /* Eq. 17 */
    T e = mj * I.A * dWi * vr;               /* Eq. 18 */
    acc_s += ps;
    a.du += e;
    if (scales) a.su += abs_(e);
  }
  if (terms & 2) {
    T mu = min0_(vr);                                         /* Eq. 11 */
    T vsig = I.c + J.c - beta * mu;                           /* Eq. 10 */
    T alpha = T(0.5) * (I.av + J.av) * (T(0.5) * (I.B + J.B)); /* Eq. 16 */
    T nu = -alpha * mu * vsig / (I.rho + J.rho);              /* Eq. 9 (reading) */
    T vs = mj * nu * T(0.5) * fsum;                           /* Eq. 7 */
    T e = T(0.5) * vs * vr;                                   /* viscous heating */
    acc_s += vs;
    a.du += e;
    if (scales) a.su += abs_(e);
  }
  if (terms & 4) {
    T Psum = I.P + J.P;
    T alpha_c = (Psum > T(0.0)) ? (I.P * I.ac + J.P * J.ac) / Psum : T(0.0); /* Eq. 20 */
    T rhos = I.rho + J.rho;
    T vc = abs_(vr) + sqrt_(T(2.0) * abs_(I.P - J.P) / rhos);               /* Eq. 22 */
    T e = alpha_c * vc * mj * (I.u - J.u) * fsum / rhos;                     /* Eq. 19 */
    a.du += e;
    if (scales) a.su += abs_(e);
  }
  a.ax -= acc_s * ex;
  a.ay -= acc_s * ey;
  a.az -= acc_s * ez;
  if (scales) a.sa += abs_(acc_s);
  a.dh += mj * dWi * vr; /* sum_j m_j v_ij . G_i */
}

int nthreads_of(const oracle_params& p) {
#ifdef _OPENMP
  return p.nthreads > 0 ? p.nthreads : omp_get_max_threads();
#else
  (void)p;
  return 1;
#endif
}

Geo geo_of(const oracle_params& p) {
  Geo g;
  for (int a = 0; a < 3; ++a) g.L[a] = p.box[a];
  g.periodic = p.periodic;
  return g;
}

double max_of(int64_t n, const double* h) {
  double hm = 0.0;
  for (int64_t i = 0; i < n; ++i) hm = std::max(hm, h[i]);
  return hm;
}

}  // namespace

extern "C" {

/* Cell id per particle (exact integer definition, see header). */
int oracle_cell_ids(int64_t n, const double* x, const double* box, int nc, uint32_t* out) {
  if (nc < 1) return -1;
  for (int64_t i = 0; i < n; ++i) {
    int cx = cell_coord(x[3 * i + 0], box[0], nc);
    int cy = cell_coord(x[3 * i + 1], box[1], nc);
    int cz = cell_coord(x[3 * i + 2], box[2], nc);
    out[i] = (uint32_t)(cx + nc * (cy + nc * cz));
  }
  return 0;
}

/* Kernel W(r,h) and dW/dr for a vector of r at one h (for the kernel pins). */
int oracle_kernel(int64_t n, const double* r, double h, double kernel_gamma, int kind, double* W, double* dWdr) {
  if (kind < 0 || kind > 2) return -1;
  KernelI<double> k = kernel_consts<double>(h, kernel_gamma, kind);
  for (int64_t i = 0; i < n; ++i) kernel_eval(k, r[i], W[i], dWdr[i]);
  return 0;
}

/*
 * Density loop at fixed h (Eq. 2-6): outputs for each i with active[i] != 0
 * (all when active == NULL); other entries are left untouched.
 */
int oracle_density(const oracle_params* p, int64_t n, const double* x, const double* v, const double* m,
                   const double* h, const uint8_t* active, double* n_out, double* dn_dh, double* rho,
                   double* drho_dh, double* div, double* curl, int64_t* ngb) {
  Geo g = geo_of(*p);
  Cells c = make_cells(g, n, x, p->kernel_gamma * max_of(n, h), p->use_cells);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads_of(*p))
  for (int64_t i = 0; i < n; ++i) {
    if (active && !active[i]) continue;
    DensOut d = density_at(g, c, n, x, v, m, i, h[i], p->kernel_gamma, p->kernel);
    if (n_out) n_out[i] = d.n;
    if (dn_dh) dn_dh[i] = d.dn_dh;
    if (rho) rho[i] = d.rho;
    if (drho_dh) drho_dh[i] = d.drho_dh;
    if (div) div[i] = d.div;
    if (curl) for (int a = 0; a < 3; ++a) curl[3 * i + a] = d.curl[a];
    if (ngb) ngb[i] = d.count;
  }
  return 0;
}

/*
 * Newton iteration on h for active particles, then the density outputs at the
 * final h. Requires h_max > 0 when use_cells is set (the cell width must cover
 * the largest support the iteration may reach).
 */
int oracle_solve_h(const oracle_params* p, int64_t n, const double* x, const double* v, const double* m,
                   const double* h_in, const uint8_t* active, double* h_out, int32_t* iters,
                   int32_t* converged, double* n_out, double* dn_dh, double* rho, double* drho_dh,
                   double* div, double* curl, int64_t* ngb, int64_t* pass_pairs) {
  Geo g = geo_of(*p);
  double rmax = p->h_max > 0 ? p->kernel_gamma * p->h_max : 0.0;
  Cells c = make_cells(g, n, x, rmax, p->use_cells && p->h_max > 0);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads_of(*p))
  for (int64_t i = 0; i < n; ++i) {
    if (active && !active[i]) {
      h_out[i] = h_in[i];
      continue;
    }
    SolveOut s = solve_h(g, c, n, x, v, m, i, h_in[i], *p);
    h_out[i] = s.h;
    if (iters) iters[i] = s.iters;
    if (converged) converged[i] = s.converged;
    if (n_out) n_out[i] = s.d.n;
    if (dn_dh) dn_dh[i] = s.d.dn_dh;
    if (rho) rho[i] = s.d.rho;
    if (drho_dh) drho_dh[i] = s.d.drho_dh;
    if (div) div[i] = s.d.div;
    if (curl) for (int a = 0; a < 3; ++a) curl[3 * i + a] = s.d.curl[a];
    if (ngb) ngb[i] = s.d.count;
    if (pass_pairs) pass_pairs[i] = s.pairs;
  }
  return 0;
}

/* Ghost step (per particle): Omega, f = 1/Omega (Eq. 8), P, c, Balsara B. */
int oracle_ghost(const oracle_params* p, int64_t n, const double* h, const double* rho,
                 const double* drho_dh, const double* div, const double* curl, const double* u,
                 double* f, double* P, double* c, double* B) {
  const double ga = p->gamma_eos;
  for (int64_t i = 0; i < n; ++i) {
    double omega = 1.0 + h[i] / (3.0 * rho[i]) * drho_dh[i];
    f[i] = 1.0 / omega;
    P[i] = (ga - 1.0) * rho[i] * u[i];
    c[i] = std::sqrt(ga * (ga - 1.0) * u[i]);
    double ad = std::fabs(div[i]);
    double ac = std::sqrt(curl[3 * i] * curl[3 * i] + curl[3 * i + 1] * curl[3 * i + 1] +
                          curl[3 * i + 2] * curl[3 * i + 2]);
    B[i] = ad > 0.0 ? ad / (ad + ac + 1e-4 * c[i] / h[i]) : 0.0;
  }
  return 0;
}

/* Gradient loop: v_sig,max (Eq. 10-11, j in N_i and i) and the Laplacian of u. */
int oracle_gradient(const oracle_params* p, int64_t n, const double* x, const double* v, const double* m,
                    const double* h, const double* rho, const double* c, const double* u,
                    const uint8_t* active, double* vsig, double* lapu) {
  Geo g = geo_of(*p);
  Cells cl = make_cells(g, n, x, p->kernel_gamma * max_of(n, h), p->use_cells);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads_of(*p))
  for (int64_t i = 0; i < n; ++i) {
    if (active && !active[i]) continue;
    KernelI<double> k = kernel_consts<double>(h[i], p->kernel_gamma, p->kernel);
    double H2 = k.H * k.H;
    GradAcc<double> a{2.0 * c[i], 0.0}; /* j = i: mu = 0 */
    for_candidates(cl, n, i, [&](int64_t j) {
      if (j == i) return;
      double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
      min_image(g, d);
      double r2 = r2_of(d);
      if (!(r2 < H2)) return;
      gradient_pair<double>(k, r2, d[0], d[1], d[2], v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1],
                            v[3 * i + 2] - v[3 * j + 2], c[i], c[j], m[j], rho[j], u[i] - u[j],
                            p->beta_v, a);
    });
    vsig[i] = a.vsig;
    lapu[i] = 2.0 * a.lap;
  }
  return 0;
}

/*
 * Force loop (Eq. 7, 9-11, 16-20, 22 with the readings in the header).
 * accel is n*3. alpha_v_i / alpha_c_i may be NULL (constants from params).
 */
int oracle_force(const oracle_params* p, int64_t n, const double* x, const double* v, const double* m,
                 const double* h, const double* u, const double* rho, const double* f, const double* P,
                 const double* c, const double* B, const double* alpha_v_i, const double* alpha_c_i,
                 const uint8_t* active, double* accel, double* dudt, double* dhdt, double* s_a,
                 double* s_u, int64_t* npairs) {
  Geo g = geo_of(*p);
  Cells cl = make_cells(g, n, x, p->kernel_gamma * max_of(n, h), p->use_cells);
  auto per = [&](int64_t i) {
    ForceI<double> I;
    I.k = kernel_consts<double>(h[i], p->kernel_gamma, p->kernel);
    I.f = f[i];
    I.rho = rho[i];
    I.P = P[i];
    I.A = f[i] * P[i] / (rho[i] * rho[i]);
    I.c = c[i];
    I.B = B[i];
    I.av = alpha_v_i ? alpha_v_i[i] : p->alpha_v;
    I.ac = alpha_c_i ? alpha_c_i[i] : p->alpha_c;
    I.u = u[i];
    return I;
  };
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads_of(*p))
  for (int64_t i = 0; i < n; ++i) {
    if (active && !active[i]) continue;
    ForceI<double> I = per(i);
    ForceAcc<double> a{0, 0, 0, 0, 0, 0, 0};
    long long cnt = 0;
    for_candidates(cl, n, i, [&](int64_t j) {
      if (j == i) return;
      double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
      min_image(g, d);
      double r2 = r2_of(d);
      double Hj = p->kernel_gamma * h[j];
      if (!(r2 < I.k.H * I.k.H) && !(r2 < Hj * Hj)) return;
      ForceI<double> J = per(j);
      force_pair<double>(I, J, r2, d[0], d[1], d[2], v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1],
                         v[3 * i + 2] - v[3 * j + 2], m[j], p->beta_v, p->terms, true, a);
      cnt++;
    });
    accel[3 * i] = a.ax;
    accel[3 * i + 1] = a.ay;
    accel[3 * i + 2] = a.az;
    dudt[i] = a.du;
    if (dhdt) dhdt[i] = -(h[i] / (3.0 * rho[i])) * f[i] * a.dh;
    if (s_a) s_a[i] = a.sa;
    if (s_u) s_u[i] = a.su;
    if (npairs) npairs[i] = cnt;
  }
  return 0;
}

/* SPH interpolant, Eq. 1: Qhat_i = sum_j (m_j/rho_j) Q_j W_ij (self included), r < H_i. */
int oracle_interpolate(const oracle_params* p, int64_t n, const double* x, const double* m,
                       const double* h, const double* rho, const double* Q, double* Qhat) {
  Geo g = geo_of(*p);
  Cells cl = make_cells(g, n, x, p->kernel_gamma * max_of(n, h), p->use_cells);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads_of(*p))
  for (int64_t i = 0; i < n; ++i) {
    KernelI<double> k = kernel_consts<double>(h[i], p->kernel_gamma, p->kernel);
    double H2 = k.H * k.H, s = 0.0;
    for_candidates(cl, n, i, [&](int64_t j) {
      double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
      min_image(g, d);
      double r2 = (j == i) ? 0.0 : r2_of(d);
      if (j != i && !(r2 < H2)) return;
      double W, dW;
      kernel_eval(k, std::sqrt(r2), W, dW);
      s += m[j] / rho[j] * Q[j] * W;
    });
    Qhat[i] = s;
  }
  return 0;
}

/*
 * Flop count of one interaction of each loop, from the same templated pair
 * functions instantiated on the counting scalar. loop: 0 density (non-self
 * hit), 1 gradient, 2 force (all terms), 3 one step of the h iteration
 * (Eqs. 5-6 only); q selects the spline branch
 * (q < 1/2 or q >= 1/2) of the i-side kernel; approaching selects the
 * mu < 0 branch. out[0..4] = add, mul, div, sqrt, cmp. The neighbour test
 * itself (3 sub, 3 mul, 2 add, 1 cmp) is not included.
 */
int oracle_count_flops(int loop, double q, int approaching, int kind, long long* out) {
  OpTally t{0, 0, 0, 0, 0};
  double h = 0.02, kg = 1.825742;
  if (kind < 0 || kind > 2) return -1;
  KernelI<Cnt> k = kernel_consts<Cnt>(h, kg, kind);
  double r = q * kg * h;
  Cnt dx(r), dy(0.0), dz(0.0), r2(r * r);
  Cnt dvx(approaching ? -0.3 : 0.3), dvy(0.1), dvz(0.2);
  g_tally = &t;
  if (loop == 0) {
    DensAcc<Cnt> a{0, 0, 0, 0, 0, 0, 0, 0, 0};
    density_pair<Cnt>(k, r2, dx, dy, dz, Cnt(1.0), dvx, dvy, dvz, false, a);
  } else if (loop == 3) {
    Cnt nn(0.0), dn(0.0);
    number_pair<Cnt>(k, r2, nn, dn);
  } else if (loop == 1) {
    GradAcc<Cnt> a{Cnt(0.0), Cnt(0.0)};
    gradient_pair<Cnt>(k, r2, dx, dy, dz, dvx, dvy, dvz, Cnt(1.0), Cnt(1.1), Cnt(1.0), Cnt(1.0),
                       Cnt(0.5), Cnt(3.0), a);
  } else {
    ForceI<Cnt> I, J;
    I.k = k;
    J.k = kernel_consts<Cnt>(h * 1.05, kg, kind);
    I.f = J.f = Cnt(1.0);
    I.A = J.A = Cnt(1.0);
    I.rho = J.rho = Cnt(1.0);
    I.P = Cnt(1.0);
    J.P = Cnt(2.0);
    I.c = J.c = Cnt(1.0);
    I.B = J.B = Cnt(0.5);
    I.av = J.av = Cnt(1.0);
    I.ac = J.ac = Cnt(1.0);
    I.u = Cnt(1.0);
    J.u = Cnt(2.0);
    ForceAcc<Cnt> a{0, 0, 0, 0, 0, 0, 0};
    force_pair<Cnt>(I, J, r2, dx, dy, dz, dvx, dvy, dvz, Cnt(1.0), Cnt(3.0), 7, false, a);
  }
  g_tally = nullptr;
  out[0] = t.add;
  out[1] = t.mul;
  out[2] = t.div;
  out[3] = t.sqrt;
  out[4] = t.cmp;
  return 0;
}

}  // extern "C"
