// FP64 CPU oracle for Gauss-Newton bundle adjustment over the DPVO patch graph.
//
// TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
// and the benchmark's CPU-baseline leg may load this library.  It shares no
// code, header, table or constant with the CUDA path.
//
// What it computes (arxiv 2408.01654, Sec. 3.1 "DPVO Preliminaries"):
//   Eq. 2  reprojection  P'_ikj = Pi[ G_j^-1 G_i Pi^-1(P_ik) ]
//   Eq. 3  argmin_{G,d} sum_(i,k,j) || P'_ikj - I_ikj ||^2_{Sigma},  Sigma = diag(w)
// solved by plain Gauss-Newton, with the inverse depths Schur-eliminated and
// the pose system Cholesky-factored (the block-sparse BA of Sec. 3.2
// "Efficient Global Optimization" and the appendix "Bundle-Adjustment
// Efficiency", which names the pose-block Cholesky of the Schur complement).
//
// Readings of points the paper leaves open (each also listed in the design
// notes of the repository):
//   * residual on the patch centre pixel only: r = I - proj (2-vector per edge);
//   * cost = sum_c w_c r_c^2 (w multiplies, Eq. 3 with Sigma = diag(w));
//   * poses stored world->camera, T_i = G_i^-1, as (t, q) with q = (x,y,z,w);
//     perturbation on the left, T <- Exp(xi) T, xi = (rho, phi) translation first;
//   * an edge is masked when i == j or when the reprojected point's depth in
//     frame j, Z/d, is below z_min (i.e. Z <= z_min * d);
//   * damping: lambda_p on every free-pose diagonal, lambda_d added to each
//     depth diagonal; pure GN, no step rejection;
//   * inverse depths clamped below at d_min after each step; the new depth is
//     written to all nine pixels of the patch.
//
// Every routine is templated on the scalar so the same plain code runs on
// forward-mode dual numbers (exact derivatives for the gradient oracle).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <vector>

namespace {

// ----------------------------------------------------------------------------
// forward-mode dual numbers (value, derivative along one seed direction)
// ----------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return {s, a.d / (2.0 * s)}; }
inline Dual sin(Dual a) { return {std::sin(a.v), a.d * std::cos(a.v)}; }
inline Dual cos(Dual a) { return {std::cos(a.v), -a.d * std::sin(a.v)}; }
inline double sqrt(double a) { return std::sqrt(a); }
inline double sin(double a) { return std::sin(a); }
inline double cos(double a) { return std::cos(a); }
inline double val(double x) { return x; }
inline double val(Dual x) { return x.v; }

// ----------------------------------------------------------------------------
// rotations and poses
// ----------------------------------------------------------------------------
template <class T> struct Pose { T t[3]; T q[4]; };  // world->camera, q=(x,y,z,w)

template <class T> void quat_to_rot(const T q[4], T R[9]) {
  const T x = q[0], y = q[1], z = q[2], w = q[3];
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - z * w);       R[2] = 2.0 * (x * z + y * w);
  R[3] = 2.0 * (x * y + z * w);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - x * w);
  R[6] = 2.0 * (x * z - y * w);       R[7] = 2.0 * (y * z + x * w);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

template <class T> void quat_mul(const T a[4], const T b[4], T c[4]) {  // c = a (x) b
  c[0] = a[3] * b[0] + a[0] * b[3] + a[1] * b[2] - a[2] * b[1];
  c[1] = a[3] * b[1] - a[0] * b[2] + a[1] * b[3] + a[2] * b[0];
  c[2] = a[3] * b[2] + a[0] * b[1] - a[1] * b[0] + a[2] * b[3];
  c[3] = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
}

// T <- Exp(xi) T with xi = (rho, phi):  Exp(xi) = [ R(phi)  V(phi) rho ; 0 1 ],
// R(phi) by the unit quaternion (sin(th/2) phi/th, cos(th/2)),
// V = I + B [phi]x + C [phi]x^2,  B = (1-cos th)/th^2,  C = (th - sin th)/th^3.
// Below th = 1e-3 every coefficient is its Taylor series in th^2 (exact to
// FP64 there); above, B is evaluated as 2 sin^2(th/2)/th^2 to avoid cancellation.
template <class T> void se3_retract(const T xi[6], Pose<T>& p) {
  const T* rho = xi;
  const T* phi = xi + 3;
  const T th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  T a, c, B, C;  // a = sin(th/2)/th, c = cos(th/2)
  if (val(th2) < 1e-6) {
    const T th4 = th2 * th2;
    a = 0.5 - th2 / 48.0 + th4 / 3840.0;
    c = 1.0 - th2 / 8.0 + th4 / 384.0;
    B = 0.5 - th2 / 24.0 + th4 / 720.0;
    C = 1.0 / 6.0 - th2 / 120.0 + th4 / 5040.0;
  } else {
    const T th = sqrt(th2);
    const T sh = sin(th * 0.5);
    a = sh / th;
    c = cos(th * 0.5);
    B = 2.0 * sh * sh / th2;
    C = (th - sin(th)) / (th2 * th);
  }
  const T qe[4] = {a * phi[0], a * phi[1], a * phi[2], c};
  // V rho = rho + B (phi x rho) + C (phi x (phi x rho))
  T pxr[3] = {phi[1] * rho[2] - phi[2] * rho[1], phi[2] * rho[0] - phi[0] * rho[2],
              phi[0] * rho[1] - phi[1] * rho[0]};
  T pxpxr[3] = {phi[1] * pxr[2] - phi[2] * pxr[1], phi[2] * pxr[0] - phi[0] * pxr[2],
                phi[0] * pxr[1] - phi[1] * pxr[0]};
  T Re[9];
  quat_to_rot(qe, Re);
  T tn[3];
  for (int r = 0; r < 3; ++r)
    tn[r] = Re[3 * r] * p.t[0] + Re[3 * r + 1] * p.t[1] + Re[3 * r + 2] * p.t[2] + rho[r] +
            B * pxr[r] + C * pxpxr[r];
  T qn[4];
  quat_mul(qe, p.q, qn);
  const T nrm = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
  for (int r = 0; r < 3; ++r) p.t[r] = tn[r];
  for (int r = 0; r < 4; ++r) p.q[r] = qn[r] / nrm;
}

// ----------------------------------------------------------------------------
// per-edge reprojection, residual and Jacobians (Eq. 2 and Eq. 3)
// ----------------------------------------------------------------------------
template <class T> struct EdgeTerms {
  T X[3];  // the point in frame j, homogeneous with last coordinate d: X / d in metres
  T proj[2], r[2];
  T Ji[2][6], Jj[2][6], Jd[2];
  bool valid;
};

template <class T>
void edge_terms(const Pose<T>& Pi, const Pose<T>& Pj, T u, T v, T d, const T tgt[2],
                const double K[4], double z_min, bool self_edge, EdgeTerms<T>& o) {
  const double fx = K[0], fy = K[1], cx = K[2], cy = K[3];
  T Ri[9], Rj[9], R[9], t[3];
  quat_to_rot(Pi.q, Ri);
  quat_to_rot(Pj.q, Rj);
  // T_ij = T_j T_i^-1 :  R = Rj Ri^T,  t = tj - R ti
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      R[3 * r + c] = Rj[3 * r] * Ri[3 * c] + Rj[3 * r + 1] * Ri[3 * c + 1] + Rj[3 * r + 2] * Ri[3 * c + 2];
  for (int r = 0; r < 3; ++r)
    t[r] = Pj.t[r] - (R[3 * r] * Pi.t[0] + R[3 * r + 1] * Pi.t[1] + R[3 * r + 2] * Pi.t[2]);
  // back-projection with inverse depth: homogeneous (x, y, 1, d)
  const T xb[3] = {(u - cx) / fx, (v - cy) / fy, T(1.0)};
  T X[3];
  for (int r = 0; r < 3; ++r) X[r] = R[3 * r] * xb[0] + R[3 * r + 1] * xb[1] + R[3 * r + 2] * xb[2] + t[r] * d;
  for (int r = 0; r < 3; ++r) o.X[r] = X[r];
  o.valid = !self_edge && val(X[2]) > z_min * val(d);
  const T iz = 1.0 / X[2];
  o.proj[0] = fx * X[0] * iz + cx;
  o.proj[1] = fy * X[1] * iz + cy;
  o.r[0] = tgt[0] - o.proj[0];
  o.r[1] = tgt[1] - o.proj[1];
  // D = d proj / d X
  const T D[2][3] = {{fx * iz, T(0.0), -fx * X[0] * iz * iz}, {T(0.0), fy * iz, -fy * X[1] * iz * iz}};
  // dX/dxi_j = [ d I | -[X]x ]
  const T M[3][6] = {{d, T(0.0), T(0.0), T(0.0), X[2], -X[1]},
                     {T(0.0), d, T(0.0), -X[2], T(0.0), X[0]},
                     {T(0.0), T(0.0), d, X[1], -X[0], T(0.0)}};
  // Ad(T_ij) = [ R  [t]x R ; 0  R ]
  T tx[9] = {T(0.0), -t[2], t[1], t[2], T(0.0), -t[0], -t[1], t[0], T(0.0)};
  T txR[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      txR[3 * r + c] = tx[3 * r] * R[c] + tx[3 * r + 1] * R[3 + c] + tx[3 * r + 2] * R[6 + c];
  T Ad[6][6];
  for (int r = 0; r < 6; ++r)
    for (int c = 0; c < 6; ++c) Ad[r][c] = T(0.0);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      Ad[r][c] = R[3 * r + c];
      Ad[r][3 + c] = txR[3 * r + c];
      Ad[3 + r][3 + c] = R[3 * r + c];
    }
  for (int a = 0; a < 2; ++a) {
    for (int c = 0; c < 6; ++c) {
      T s = T(0.0);
      for (int m = 0; m < 3; ++m) s += D[a][m] * M[m][c];
      o.Jj[a][c] = s;
    }
    for (int c = 0; c < 6; ++c) {
      T s = T(0.0);
      for (int m = 0; m < 6; ++m) s += o.Jj[a][m] * Ad[m][c];
      o.Ji[a][c] = -s;
    }
    o.Jd[a] = D[a][0] * t[0] + D[a][1] * t[1] + D[a][2] * t[2];
  }
}

// ----------------------------------------------------------------------------
// problem description shared by the entry points
// ----------------------------------------------------------------------------
struct Opts { double lambda_p, lambda_d, z_min, d_min; };

template <class T> struct Problem {
  int N, P, E;
  int pix = 1;                     // residual pixels per edge: 1 (the centre) or 9 (the whole patch)
  std::vector<Pose<T>> poses;      // [N]
  std::vector<T> u, v, d;          // patch centre pixel and inverse depth [P]
  std::vector<T> pu, pv;           // all nine pixels of each patch [P,9] (row-major 3x3)
  const int *ii, *jj, *kk;
  std::vector<T> tgt, wgt;         // [E,pix,2], [E,2]
  double K[4];
  // pixel q of the edge's residual: the centre (4) when pix = 1
  int pixel(int q) const { return pix == 1 ? 4 : q; }
};

template <class T>
void load_problem(Problem<T>& pb, int N, int P, int E, const double* poses, const double* patches,
                  const int* ii, const int* jj, const int* kk, const double* targets,
                  const double* weights, const double* intr, int pix = 1) {
  pb.N = N; pb.P = P; pb.E = E;
  pb.pix = pix;
  pb.poses.resize(N);
  for (int a = 0; a < N; ++a) {
    for (int r = 0; r < 3; ++r) pb.poses[a].t[r] = T(poses[7 * a + r]);
    for (int r = 0; r < 4; ++r) pb.poses[a].q[r] = T(poses[7 * a + 3 + r]);
  }
  pb.u.resize(P); pb.v.resize(P); pb.d.resize(P);
  for (int k = 0; k < P; ++k) {  // patches [P,3,3,3]: centre pixel is [k][c][1][1]
    pb.u[k] = T(patches[27 * k + 0 * 9 + 4]);
    pb.v[k] = T(patches[27 * k + 1 * 9 + 4]);
    pb.d[k] = T(patches[27 * k + 2 * 9 + 4]);
  }
  pb.pu.resize(9 * (size_t)P); pb.pv.resize(9 * (size_t)P);
  for (int k = 0; k < P; ++k)
    for (int q = 0; q < 9; ++q) {
      pb.pu[9 * (size_t)k + q] = T(patches[27 * k + q]);
      pb.pv[9 * (size_t)k + q] = T(patches[27 * k + 9 + q]);
    }
  pb.ii = ii; pb.jj = jj; pb.kk = kk;
  pb.tgt.resize(2 * (size_t)E * pix); pb.wgt.resize(2 * (size_t)E);
  for (size_t e = 0; e < 2 * (size_t)E * pix; ++e) pb.tgt[e] = T(targets[e]);
  for (size_t e = 0; e < 2 * (size_t)E; ++e) pb.wgt[e] = T(weights[e]);
  for (int r = 0; r < 4; ++r) pb.K[r] = intr[r];
}

int check_indices(int N, int P, int E, const int* ii, const int* jj, const int* kk) {
  std::vector<int> src(P, -1);
  for (int e = 0; e < E; ++e) {
    if (ii[e] < 0 || ii[e] >= N || jj[e] < 0 || jj[e] >= N || kk[e] < 0 || kk[e] >= P) return 1;
    if (src[kk[e]] < 0) src[kk[e]] = ii[e];
    else if (src[kk[e]] != ii[e]) return 1;  // one source frame per patch
  }
  return 0;
}

// ----------------------------------------------------------------------------
// normal equations with the inverse depths eliminated (Schur complement)
//   H = [ B  E ; E^T  C ],  g = [ v ; w ],  r ~ r - J delta  =>  H delta = g
//   S = B + lambda_p I - E Ct^-1 E^T,   y = v - E Ct^-1 w,   Ct = C + lambda_d
// Only free poses (index >= fixed) are variables.
// ----------------------------------------------------------------------------
template <class T> struct Linear {
  int n;                                   // 6 * free poses
  std::vector<T> B, vv;                    // dense [n*n], [n]
  std::vector<T> C, w;                     // [P]
  std::vector<std::vector<std::pair<int, std::vector<T>>>> Ek;  // per patch: (free pose, 6-vector)
  T cost;
};

template <class T> std::vector<T>& ek_slot(std::vector<std::pair<int, std::vector<T>>>& lst, int a) {
  for (auto& pr : lst)
    if (pr.first == a) return pr.second;
  lst.emplace_back(a, std::vector<T>(6, T(0.0)));
  return lst.back().second;
}

template <class T>
void linearize(const Problem<T>& pb, int fixed, const Opts& o, Linear<T>& L) {
  const int nf = pb.N - fixed;
  L.n = 6 * nf;
  L.B.assign((size_t)L.n * L.n, T(0.0));
  L.vv.assign(L.n, T(0.0));
  L.C.assign(pb.P, T(0.0));
  L.w.assign(pb.P, T(0.0));
  L.Ek.assign(pb.P, {});
  L.cost = T(0.0);
  EdgeTerms<T> et;
  // each edge contributes one 2-D residual per residual pixel (Eq. 3 sums
  // over the patch's pixels; with pix = 1 only its centre), all with the
  // edge's weight
  for (int e = 0; e < pb.E; ++e)  // input order
   for (int q = 0; q < pb.pix; ++q) {
    const int i = pb.ii[e], j = pb.jj[e], k = pb.kk[e];
    const size_t px = 9 * (size_t)k + pb.pixel(q);
    edge_terms(pb.poses[i], pb.poses[j], pb.pu[px], pb.pv[px], pb.d[k], &pb.tgt[2 * ((size_t)e * pb.pix + q)],
               pb.K, o.z_min, i == j, et);
    if (!et.valid) continue;
    const T* w = &pb.wgt[2 * (size_t)e];
    for (int c = 0; c < 2; ++c) L.cost += w[c] * et.r[c] * et.r[c];
    const int fi = i - fixed, fj = j - fixed;  // free index or negative
    // depth-depth and depth-gradient
    for (int c = 0; c < 2; ++c) {
      L.C[k] += w[c] * et.Jd[c] * et.Jd[c];
      L.w[k] += w[c] * et.Jd[c] * et.r[c];
    }
    const T* Jp[2] = {&et.Ji[0][0], &et.Jj[0][0]};
    const int fp[2] = {fi, fj};
    for (int s = 0; s < 2; ++s) {
      if (fp[s] < 0) continue;
      // pose gradient and pose-depth coupling
      std::vector<T>& Ev = ek_slot(L.Ek[k], fp[s]);
      for (int r = 0; r < 6; ++r) {
        T gv = T(0.0), ev = T(0.0);
        for (int c = 0; c < 2; ++c) {
          gv += w[c] * Jp[s][6 * c + r] * et.r[c];
          ev += w[c] * Jp[s][6 * c + r] * et.Jd[c];
        }
        L.vv[6 * fp[s] + r] += gv;
        Ev[r] += ev;
      }
      // pose-pose blocks
      for (int s2 = 0; s2 < 2; ++s2) {
        if (fp[s2] < 0) continue;
        for (int r = 0; r < 6; ++r)
          for (int cc = 0; cc < 6; ++cc) {
            T h = T(0.0);
            for (int c = 0; c < 2; ++c) h += w[c] * Jp[s][6 * c + r] * Jp[s2][6 * c + cc];
            L.B[(size_t)(6 * fp[s] + r) * L.n + 6 * fp[s2] + cc] += h;
          }
      }
    }
  }
}

template <class T>
void schur(const Problem<T>& pb, const Opts& o, Linear<T>& L, std::vector<T>& S, std::vector<T>& y) {
  const int n = L.n;
  S = L.B;
  y = L.vv;
  for (int r = 0; r < n; ++r) S[(size_t)r * n + r] += o.lambda_p;
  for (int k = 0; k < pb.P; ++k) {
    const T Ct = L.C[k] + o.lambda_d;
    for (auto& pa : L.Ek[k]) {
      for (int r = 0; r < 6; ++r) y[6 * pa.first + r] -= pa.second[r] * L.w[k] / Ct;
      for (auto& pb2 : L.Ek[k])
        for (int r = 0; r < 6; ++r)
          for (int c = 0; c < 6; ++c)
            S[(size_t)(6 * pa.first + r) * n + 6 * pb2.first + c] -= pa.second[r] * pb2.second[c] / Ct;
    }
  }
}

// plain dense Cholesky S = L L^T (lower, in place) and the two triangular solves
template <class T> int cholesky_solve(std::vector<T>& S, int n, const std::vector<T>& y, std::vector<T>& x) {
  for (int j = 0; j < n; ++j) {
    T s = S[(size_t)j * n + j];
    for (int p = 0; p < j; ++p) s -= S[(size_t)j * n + p] * S[(size_t)j * n + p];
    if (!(val(s) > 0.0)) return 4;  // not positive definite
    const T ljj = sqrt(s);
    S[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      T a = S[(size_t)i * n + j];
      for (int p = 0; p < j; ++p) a -= S[(size_t)i * n + p] * S[(size_t)j * n + p];
      S[(size_t)i * n + j] = a / ljj;
    }
  }
  x = y;
  for (int i = 0; i < n; ++i) {  // L z = y
    T a = x[i];
    for (int p = 0; p < i; ++p) a -= S[(size_t)i * n + p] * x[p];
    x[i] = a / S[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {  // L^T x = z
    T a = x[i];
    for (int p = i + 1; p < n; ++p) a -= S[(size_t)p * n + i] * x[p];
    x[i] = a / S[(size_t)i * n + i];
  }
  return 0;
}

// one GN iteration: linearise, eliminate depths, solve, back-substitute, retract
template <class T>
int gn_iteration(Problem<T>& pb, int fixed, const Opts& o, std::vector<T>* dxi_out, std::vector<T>* dd_out,
                 T* cost_out) {
  Linear<T> L;
  linearize(pb, fixed, o, L);
  std::vector<T> S, y, dxi;
  schur(pb, o, L, S, y);
  const int n = L.n;
  int st = cholesky_solve(S, n, y, dxi);
  if (st) return st;
  std::vector<T> dd(pb.P, T(0.0));
  for (int k = 0; k < pb.P; ++k) {  // dd_k = Ct_k^-1 (w_k - sum_a E_ak^T dxi_a)
    T a = L.w[k];
    for (auto& pa : L.Ek[k])
      for (int r = 0; r < 6; ++r) a -= pa.second[r] * dxi[6 * pa.first + r];
    dd[k] = a / (L.C[k] + o.lambda_d);
  }
  for (int f = 0; f < pb.N - fixed; ++f) se3_retract(&dxi[6 * f], pb.poses[fixed + f]);
  for (int k = 0; k < pb.P; ++k) {
    T nd = pb.d[k] + dd[k];
    pb.d[k] = val(nd) > o.d_min ? nd : T(o.d_min);
  }
  if (dxi_out) *dxi_out = dxi;
  if (dd_out) *dd_out = dd;
  if (cost_out) *cost_out = L.cost;
  return 0;
}

template <class T>
T problem_cost(const Problem<T>& pb, const Opts& o) {
  T cost = T(0.0);
  EdgeTerms<T> et;
  for (int e = 0; e < pb.E; ++e)
    for (int q = 0; q < pb.pix; ++q) {
      const int i = pb.ii[e], j = pb.jj[e], k = pb.kk[e];
      const size_t px = 9 * (size_t)k + pb.pixel(q);
      edge_terms(pb.poses[i], pb.poses[j], pb.pu[px], pb.pv[px], pb.d[k], &pb.tgt[2 * ((size_t)e * pb.pix + q)],
                 pb.K, o.z_min, i == j, et);
      if (!et.valid) continue;
      for (int c = 0; c < 2; ++c) cost += pb.wgt[2 * (size_t)e + c] * et.r[c] * et.r[c];
    }
  return cost;
}

void store_state(const Problem<double>& pb, double* poses, double* patches) {
  for (int a = 0; a < pb.N; ++a) {
    for (int r = 0; r < 3; ++r) poses[7 * a + r] = pb.poses[a].t[r];
    for (int r = 0; r < 4; ++r) poses[7 * a + 3 + r] = pb.poses[a].q[r];
  }
  for (int k = 0; k < pb.P; ++k)
    for (int p = 0; p < 9; ++p) patches[27 * k + 18 + p] = pb.d[k];
}

}  // namespace

// ============================================================================
// C entry points (ctypes).  All arrays are host memory, row-major, float64
// unless stated; indices int32.  Return 0 on success, 1 on bad indices,
// 4 if the reduced pose system is not positive definite.
// ============================================================================
extern "C" {

int oracle_version() { return 1; }

void oracle_se3_retract(const double* xi, const double* pose_in, double* pose_out) {
  Pose<double> p;
  for (int r = 0; r < 3; ++r) p.t[r] = pose_in[r];
  for (int r = 0; r < 4; ++r) p.q[r] = pose_in[3 + r];
  se3_retract(xi, p);
  for (int r = 0; r < 3; ++r) pose_out[r] = p.t[r];
  for (int r = 0; r < 4; ++r) pose_out[3 + r] = p.q[r];
}

void oracle_quat_to_rot(const double* q, double* R) { quat_to_rot(q, R); }

// per-edge projection, Jacobians (Ji, Jj [E,2,6], Jd [E,2]) and validity
int oracle_edge_terms(int N, int P, int E, const double* poses, const double* patches, const int* ii,
                      const int* jj, const int* kk, const double* targets, const double* intr, double z_min,
                      double* proj, double* res, double* Ji, double* Jj, double* Jd, int* valid) {
  if (check_indices(N, P, E, ii, jj, kk)) return 1;
  std::vector<double> ones(2 * (size_t)E, 1.0);
  Problem<double> pb;
  load_problem(pb, N, P, E, poses, patches, ii, jj, kk, targets, ones.data(), intr);
  EdgeTerms<double> et;
  for (int e = 0; e < E; ++e) {
    const int i = ii[e], j = jj[e], k = kk[e];
    edge_terms(pb.poses[i], pb.poses[j], pb.u[k], pb.v[k], pb.d[k], &pb.tgt[2 * (size_t)e], pb.K, z_min, i == j,
               et);
    for (int c = 0; c < 2; ++c) {
      proj[2 * e + c] = et.proj[c];
      res[2 * e + c] = et.r[c];
      Jd[2 * e + c] = et.Jd[c];
      for (int m = 0; m < 6; ++m) {
        Ji[12 * (size_t)e + 6 * c + m] = et.Ji[c][m];
        Jj[12 * (size_t)e + 6 * c + m] = et.Jj[c][m];
      }
    }
    valid[e] = et.valid ? 1 : 0;
  }
  return 0;
}

// reduced pose system of the current state: S [n*n] (full, symmetric), y [n],
// Ct [P] = C + lambda_d, w [P]; n = 6 (N - fixed); cost = sum w r^2
// pix = 1: one residual per edge at the patch centre, targets [E,2];
// pix = 9: one per patch pixel, targets [E,9,2] (row-major 3x3), one weight
// pair per edge shared by its nine residuals.
int oracle_schur_system_px(int N, int P, int E, const double* poses, const double* patches, const int* ii,
                           const int* jj, const int* kk, const double* targets, const double* weights,
                           const double* intr, int fixed, const double* opts4, int pix, double* S, double* y,
                           double* Ct, double* w, double* cost) {
  if (check_indices(N, P, E, ii, jj, kk) || (pix != 1 && pix != 9)) return 1;
  const Opts o{opts4[0], opts4[1], opts4[2], opts4[3]};
  Problem<double> pb;
  load_problem(pb, N, P, E, poses, patches, ii, jj, kk, targets, weights, intr, pix);
  Linear<double> L;
  linearize(pb, fixed, o, L);
  std::vector<double> Sv, yv;
  schur(pb, o, L, Sv, yv);
  std::memcpy(S, Sv.data(), Sv.size() * sizeof(double));
  std::memcpy(y, yv.data(), yv.size() * sizeof(double));
  for (int k = 0; k < P; ++k) { Ct[k] = L.C[k] + o.lambda_d; w[k] = L.w[k]; }
  *cost = L.cost;
  return 0;
}

// `iters` GN iterations in place on poses [N,7] and patches [P,3,3,3];
// dxi [iters, 6(N-fixed)], dd [iters, P], cost [iters+1] (cost before each
// iteration and after the last).
int oracle_gn_px(int N, int P, int E, double* poses, double* patches, const int* ii, const int* jj,
                 const int* kk, const double* targets, const double* weights, const double* intr, int iters,
                 int fixed, const double* opts4, int pix, double* dxi, double* dd, double* cost) {
  if (check_indices(N, P, E, ii, jj, kk) || (pix != 1 && pix != 9)) return 1;
  const Opts o{opts4[0], opts4[1], opts4[2], opts4[3]};
  Problem<double> pb;
  load_problem(pb, N, P, E, poses, patches, ii, jj, kk, targets, weights, intr, pix);
  const int n = 6 * (N - fixed);
  for (int it = 0; it < iters; ++it) {
    std::vector<double> x, dk;
    double c;
    int st = gn_iteration(pb, fixed, o, &x, &dk, &c);
    if (st) return st;
    if (dxi) std::memcpy(dxi + (size_t)it * n, x.data(), n * sizeof(double));
    if (dd) std::memcpy(dd + (size_t)it * P, dk.data(), P * sizeof(double));
    if (cost) cost[it] = c;
    store_state(pb, poses, patches);
  }
  if (cost) cost[iters] = problem_cost(pb, o);
  return 0;
}

int oracle_schur_system(int N, int P, int E, const double* poses, const double* patches, const int* ii,
                        const int* jj, const int* kk, const double* targets, const double* weights,
                        const double* intr, int fixed, const double* opts4, double* S, double* y, double* Ct,
                        double* w, double* cost) {
  return oracle_schur_system_px(N, P, E, poses, patches, ii, jj, kk, targets, weights, intr, fixed, opts4, 1, S, y,
                                Ct, w, cost);
}

int oracle_gn(int N, int P, int E, double* poses, double* patches, const int* ii, const int* jj, const int* kk,
              const double* targets, const double* weights, const double* intr, int iters, int fixed,
              const double* opts4, double* dxi, double* dd, double* cost) {
  return oracle_gn_px(N, P, E, poses, patches, ii, jj, kk, targets, weights, intr, iters, fixed, opts4, 1, dxi, dd,
                      cost);
}

// forward-mode derivative of  L = <a, poses_final> + <b, depths_final>  with
// respect to single input coordinates: kind[c] = 0 -> targets[index[c]],
// kind[c] = 1 -> weights[index[c]] (index into the flattened [E,2] array),
// kind[c] = 2 -> the initial inverse depth of patch index[c],
// kind[c] = 3 -> component m = index[c] % 6 of a left perturbation
// T <- Exp(xi) T, xi = (rho, phi), of initial pose a = index[c] / 6, whose
// first-order change is dt = rho + phi x t, dq = (phi/2, 0) (x) q.
// One dual-number GN run per coordinate.
// pix residual pixels per edge (1 or 9; targets [E,pix,2], kind 0 indexes them)
int oracle_grad_fwd_px(int N, int P, int E, const double* poses, const double* patches, const int* ii,
                       const int* jj, const int* kk, const double* targets, const double* weights,
                       const double* intr, int iters, int fixed, const double* opts4, int pix, const double* a,
                       const double* b, int ncoord, const int* kind, const long long* index, double* out) {
  if (check_indices(N, P, E, ii, jj, kk) || (pix != 1 && pix != 9)) return 1;
  const Opts o{opts4[0], opts4[1], opts4[2], opts4[3]};
  for (int c = 0; c < ncoord; ++c) {
    const long long lim = kind[c] == 0 ? 2LL * E * pix : kind[c] == 1 ? 2LL * E : (kind[c] == 2 ? (long long)P : 6LL * N);
    if (kind[c] < 0 || kind[c] > 3 || index[c] < 0 || index[c] >= lim) return 1;
  }
  for (int c = 0; c < ncoord; ++c) {
    Problem<Dual> pb;
    load_problem(pb, N, P, E, poses, patches, ii, jj, kk, targets, weights, intr, pix);
    if (kind[c] == 0) {
      pb.tgt[index[c]].d = 1.0;
    } else if (kind[c] == 1) {
      pb.wgt[index[c]].d = 1.0;
    } else if (kind[c] == 2) {
      pb.d[index[c]].d = 1.0;
    } else {
      const int a = (int)(index[c] / 6), m = (int)(index[c] % 6);
      double xi[6] = {0, 0, 0, 0, 0, 0};
      xi[m] = 1.0;
      double t[3], q[4];
      for (int r = 0; r < 3; ++r) t[r] = pb.poses[a].t[r].v;
      for (int r = 0; r < 4; ++r) q[r] = pb.poses[a].q[r].v;
      const double half_phi[4] = {0.5 * xi[3], 0.5 * xi[4], 0.5 * xi[5], 0.0};
      double dq[4];
      quat_mul(half_phi, q, dq);
      const double dt[3] = {xi[0] + xi[4] * t[2] - xi[5] * t[1], xi[1] + xi[5] * t[0] - xi[3] * t[2],
                            xi[2] + xi[3] * t[1] - xi[4] * t[0]};
      for (int r = 0; r < 3; ++r) pb.poses[a].t[r].d = dt[r];
      for (int r = 0; r < 4; ++r) pb.poses[a].q[r].d = dq[r];
    }
    for (int it = 0; it < iters; ++it) {
      int st = gn_iteration(pb, fixed, o, (std::vector<Dual>*)nullptr, (std::vector<Dual>*)nullptr,
                            (Dual*)nullptr);
      if (st) return st;
    }
    double g = 0.0;
    for (int q = 0; q < N; ++q) {
      for (int r = 0; r < 3; ++r) g += a[7 * q + r] * pb.poses[q].t[r].d;
      for (int r = 0; r < 4; ++r) g += a[7 * q + 3 + r] * pb.poses[q].q[r].d;
    }
    for (int k = 0; k < P; ++k) g += b[k] * pb.d[k].d;
    out[c] = g;
  }
  return 0;
}

int oracle_grad_fwd(int N, int P, int E, const double* poses, const double* patches, const int* ii,
                    const int* jj, const int* kk, const double* targets, const double* weights,
                    const double* intr, int iters, int fixed, const double* opts4, const double* a,
                    const double* b, int ncoord, const int* kind, const long long* index, double* out) {
  return oracle_grad_fwd_px(N, P, E, poses, patches, ii, jj, kk, targets, weights, intr, iters, fixed, opts4, 1, a,
                            b, ncoord, kind, index, out);
}

// Proximity loop edges (Sec. 3.2 "Proximity Loop Closure", "Constructing the
// Patch Graph"): loops are found from how close the camera comes to a place it
// visited before, and every loop adds uni-directional edges from the stored
// patches of the old frame to the recent frame, so that only the recent
// frame's dense features are needed.  The paper gives no numbers; the rule
// taken here, for each query frame b in [b0, b1):
//   candidates : frames a with 0 <= a and b - a > gap (strictly older);
//   distance   : Euclidean distance between camera centres c = -R^T t of the
//                world->camera poses (the camera positions in the world);
//   selection  : the nearest candidate (the lowest index among equals), kept
//                if its distance is < radius;
//   edges      : patch k = a*M + m of that frame a, for m = 0..M-1, observed in
//                frame b (ii = a, jj = b, kk = k), kept if its centre pixel
//                reprojects (Eq. 2, current inverse depth) at least z_min in
//                front of frame b and inside [0, width) x [0, height);
//   order      : by b, then m.
// Outputs: match[q] (the selected a, or -1), dist[q] (distance of the nearest
// candidate, -1 if there is none), margin[q] (the smallest distance of any of
// the query's decisions from its threshold, scaled: (second - nearest) /
// radius, |nearest - radius| / radius, |X_z - z_min d| / (|X_z| + z_min |d|),
// the reprojection's pixel distance to the image border / max(width, height);
// 1e300 when there is nothing to decide), and the first `cap` edges with their
// reprojected centres coords [.,2]; *n_out = number of edges (may exceed cap).
int oracle_proximity_edges(int N, int M, const double* poses, const double* patches, const double* intr, int b0,
                           int b1, int gap, double radius, double z_min, double width, double height, int* match,
                           double* dist, double* margin, int* ii, int* jj, int* kk, double* coords,
                           long long cap, long long* n_out) {
  if (N < 1 || M < 1 || b0 < 0 || b1 < b0 || b1 > N || gap < 0) return 1;
  std::vector<double> centre(3 * (size_t)N);
  std::vector<Pose<double>> ps(N);
  for (int a = 0; a < N; ++a) {
    for (int r = 0; r < 3; ++r) ps[a].t[r] = poses[7 * (size_t)a + r];
    for (int r = 0; r < 4; ++r) ps[a].q[r] = poses[7 * (size_t)a + 3 + r];
    double R[9];
    quat_to_rot(ps[a].q, R);
    for (int c = 0; c < 3; ++c)  // (R^T t)_c = sum_r R[r][c] t[r]
      centre[3 * (size_t)a + c] = -(R[c] * ps[a].t[0] + R[3 + c] * ps[a].t[1] + R[6 + c] * ps[a].t[2]);
  }
  long long n = 0;
  const double tgt0[2] = {0.0, 0.0};
  for (int b = b0; b < b1; ++b) {
    const int q = b - b0;
    int best = -1;
    double d1 = 0.0, d2 = -1.0;  // nearest and second-nearest candidate distances
    for (int a = 0; a < b - gap; ++a) {
      double s = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double e = centre[3 * (size_t)a + c] - centre[3 * (size_t)b + c];
        s += e * e;
      }
      const double d = std::sqrt(s);
      if (best < 0 || d < d1) {
        d2 = best < 0 ? -1.0 : d1;
        best = a;
        d1 = d;
      } else if (d2 < 0.0 || d < d2) {
        d2 = d;
      }
    }
    double mg = 1e300;
    match[q] = -1;
    dist[q] = best < 0 ? -1.0 : d1;
    if (best >= 0) {
      mg = std::min(mg, std::fabs(d1 - radius) / radius);
      if (d1 < radius) {
        match[q] = best;
        if (d2 >= 0.0) mg = std::min(mg, (d2 - d1) / radius);
        EdgeTerms<double> et;
        for (int m = 0; m < M; ++m) {
          const long long k = (long long)best * M + m;
          const double* pk = patches + 27 * k;
          const double u = pk[4], v = pk[9 + 4], d = pk[18 + 4];
          edge_terms(ps[best], ps[b], u, v, d, tgt0, intr, z_min, false, et);
          mg = std::min(mg, std::fabs(et.X[2] - z_min * d) / (std::fabs(et.X[2]) + z_min * std::fabs(d)));
          if (!et.valid) continue;
          const double x = et.proj[0], y = et.proj[1];
          mg = std::min(mg, std::min(std::min(std::fabs(x), std::fabs(x - width)),
                                     std::min(std::fabs(y), std::fabs(y - height))) / std::max(width, height));
          if (!(x >= 0.0 && x < width && y >= 0.0 && y < height)) continue;
          if (n < cap) {
            ii[n] = best;
            jj[n] = b;
            kk[n] = (int)k;
            coords[2 * n] = x;
            coords[2 * n + 1] = y;
          }
          ++n;
        }
      }
    }
    margin[q] = mg;
  }
  *n_out = n;
  return 0;
}

// Patch correlation (Sec. 3.1 "Patch correlation", Eq. 4):
//   C(e, v, u, a, b) = < g_kk[e](v, u), f_jj[e](P'_e(v, u) + Delta_ab) >
// for every edge e, patch pixel (row v, column u) of the p x p patch, and the
// (2R+1) x (2R+1) integer offsets Delta_ab = (b - R, a - R) (a the row offset,
// b the column offset).  g: the patch's correlation features [P, p, p, D];
// f: the target frame's dense feature map [Nf, H, W, D] (channels last);
// P': the reprojected pixel [E, p, p, 2] as (x, y) in feature-map pixels,
// integer coordinates at pixel centres.  f(x, y) is bilinear sampling from the
// four pixels around (x, y) with weights (1-ax)(1-ay), ax(1-ay), (1-ax)ay, ax ay
// (x0 = floor x, ax = x - x0, likewise y); pixels outside the map are zero.
// out [E, p, p, 2R+1, 2R+1]; bound (same shape, may be null) is the same sum
// with |g| and |f| (the scale of the rounding error of any summation order).
int oracle_patch_correlation(int Nf, int H, int W, int D, int P, int p, int E, const float* fmap,
                             const float* gmap, const int* kk, const int* jj, const float* coords, int R,
                             double* out, double* bound) {
  for (int e = 0; e < E; ++e)
    if (kk[e] < 0 || kk[e] >= P || jj[e] < 0 || jj[e] >= Nf) return 1;
  const int G = 2 * R + 1;
  auto tap = [&](int j, int y, int x) -> const float* {
    if (x < 0 || x >= W || y < 0 || y >= H) return nullptr;
    return fmap + (((size_t)j * H + y) * W + x) * D;
  };
  for (int e = 0; e < E; ++e) {
    const int j = jj[e];
    for (int v = 0; v < p; ++v)
      for (int u = 0; u < p; ++u) {
        const float* g = gmap + (((size_t)kk[e] * p + v) * p + u) * D;
        const double x = coords[(((size_t)e * p + v) * p + u) * 2];
        const double y = coords[(((size_t)e * p + v) * p + u) * 2 + 1];
        for (int a = 0; a < G; ++a)
          for (int b = 0; b < G; ++b) {
            const double sx = x + (b - R), sy = y + (a - R);
            const double fx0 = std::floor(sx), fy0 = std::floor(sy);
            const double ax = sx - fx0, ay = sy - fy0;
            const int x0 = (int)fx0, y0 = (int)fy0;
            const double wts[4] = {(1 - ax) * (1 - ay), ax * (1 - ay), (1 - ax) * ay, ax * ay};
            const int xs[4] = {x0, x0 + 1, x0, x0 + 1}, ys[4] = {y0, y0, y0 + 1, y0 + 1};
            double c = 0.0, cb = 0.0;
            for (int q = 0; q < 4; ++q) {
              const float* f = tap(j, ys[q], xs[q]);
              if (!f) continue;
              double dot = 0.0, adot = 0.0;
              for (int d = 0; d < D; ++d) {
                dot += (double)g[d] * (double)f[d];
                adot += std::fabs((double)g[d] * (double)f[d]);
              }
              c += wts[q] * dot;
              cb += wts[q] * adot;
            }
            const size_t o = ((((size_t)e * p + v) * p + u) * G + a) * G + b;
            out[o] = c;
            if (bound) bound[o] = cb;
          }
      }
  }
  return 0;
}

}  // extern "C"

namespace {
// ---------------------------------------------------------------------------
// Sim(3) pose-graph optimisation (Sec. 3.3 "Optimization", Eqs. 5-7)
// ---------------------------------------------------------------------------
// A similarity S = (q, t, s) maps x to s R(q) x + t (camera to world, as the
// paper's G_i with a scale), stored as 8 doubles (tx, ty, tz, qx, qy, qz, qw, s).
// Its tangent vector xi = (rho, phi, sigma) is the matrix [[phi]x + sigma I, rho;
// 0, 0]; Exp gives R = exp([phi]x), s = e^sigma, t = W rho with
//   W = int_0^1 exp(tau ([phi]x + sigma I)) dtau = a I + b [phi]x + c [phi]x^2,
//   a = int e^{sigma tau}, b = int e^{sigma tau} sin(theta tau) / theta,
//   c = int e^{sigma tau} (1 - cos(theta tau)) / theta^2  (tau over [0, 1]).
struct Sim3 {
  double q[4], t[3], s;
};

Sim3 sim3_load(const double* v) {
  Sim3 S;
  for (int k = 0; k < 3; ++k) S.t[k] = v[k];
  for (int k = 0; k < 4; ++k) S.q[k] = v[3 + k];
  S.s = v[7];
  return S;
}

void sim3_store(const Sim3& S, double* v) {
  for (int k = 0; k < 3; ++k) v[k] = S.t[k];
  for (int k = 0; k < 4; ++k) v[3 + k] = S.q[k];
  v[7] = S.s;
}

void rot_apply(const double q[4], const double x[3], double y[3]) {
  double R[9];
  quat_to_rot(q, R);
  for (int r = 0; r < 3; ++r) y[r] = R[3 * r] * x[0] + R[3 * r + 1] * x[1] + R[3 * r + 2] * x[2];
}

Sim3 sim3_mul(const Sim3& A, const Sim3& B) {  // A B: x -> A(B(x))
  Sim3 C;
  quat_mul(A.q, B.q, C.q);
  double Rt[3];
  rot_apply(A.q, B.t, Rt);
  for (int k = 0; k < 3; ++k) C.t[k] = A.s * Rt[k] + A.t[k];
  C.s = A.s * B.s;
  return C;
}

Sim3 sim3_inv(const Sim3& A) {
  Sim3 B;
  B.q[0] = -A.q[0];
  B.q[1] = -A.q[1];
  B.q[2] = -A.q[2];
  B.q[3] = A.q[3];
  double Rt[3];
  rot_apply(B.q, A.t, Rt);
  for (int k = 0; k < 3; ++k) B.t[k] = -Rt[k] / A.s;
  B.s = 1.0 / A.s;
  return B;
}

// m_k(sigma) = int_0^1 tau^k e^{sigma tau} dtau
double moment(int k, double sg) {
  if (std::fabs(sg) < 2.0) {
    double term = 1.0, sum = 0.0;  // sum_j sigma^j / (j! (k + j + 1))
    for (int j = 0; j < 40; ++j) {
      sum += term / (k + j + 1);
      term *= sg / (j + 1);
    }
    return sum;
  }
  double m = std::expm1(sg) / sg;
  for (int i = 1; i <= k; ++i) m = (std::exp(sg) - i * m) / sg;
  return m;
}

// coefficients of W = a I + b [phi]x + c [phi]x^2
void w_coeffs(double th, double sg, double& a, double& b, double& c) {
  a = moment(0, sg);
  if (th < 1e-4) {
    b = moment(1, sg) - th * th / 6.0 * moment(3, sg);
    c = moment(2, sg) / 2.0 - th * th / 24.0 * moment(4, sg);
    return;
  }
  const double es = std::exp(sg), den = sg * sg + th * th;
  b = (es * (sg * std::sin(th) - th * std::cos(th)) + th) / (th * den);
  c = (a - (es * (sg * std::cos(th) + th * std::sin(th)) - sg) / den) / (th * th);
}

void w_apply(const double phi[3], double a, double b, double c, const double x[3], double y[3]) {
  const double px[3] = {phi[1] * x[2] - phi[2] * x[1], phi[2] * x[0] - phi[0] * x[2], phi[0] * x[1] - phi[1] * x[0]};
  const double ppx[3] = {phi[1] * px[2] - phi[2] * px[1], phi[2] * px[0] - phi[0] * px[2],
                         phi[0] * px[1] - phi[1] * px[0]};
  for (int k = 0; k < 3; ++k) y[k] = a * x[k] + b * px[k] + c * ppx[k];
}

Sim3 sim3_exp(const double xi[7]) {
  const double* rho = xi;
  const double* phi = xi + 3;
  const double sg = xi[6];
  const double th = std::sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
  Sim3 S;
  const double h = th < 1e-8 ? 0.5 - th * th / 48.0 : std::sin(0.5 * th) / th;  // sin(th/2)/th
  for (int k = 0; k < 3; ++k) S.q[k] = h * phi[k];
  S.q[3] = std::cos(0.5 * th);
  double a, b, c;
  w_coeffs(th, sg, a, b, c);
  w_apply(phi, a, b, c, rho, S.t);
  S.s = std::exp(sg);
  return S;
}

void sim3_log(const Sim3& S, double xi[7]) {
  double q[4] = {S.q[0], S.q[1], S.q[2], S.q[3]};
  if (q[3] < 0.0)
    for (double& v : q) v = -v;
  const double vn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  const double th = 2.0 * std::atan2(vn, q[3]);
  const double f = vn > 1e-12 ? th / vn : 2.0 / q[3];
  double* phi = xi + 3;
  for (int k = 0; k < 3; ++k) phi[k] = f * q[k];
  const double sg = std::log(S.s);
  xi[6] = sg;
  double a, b, c;
  w_coeffs(th, sg, a, b, c);
  // W as a 3x3 matrix, then rho = W^-1 t (adjugate)
  double Wm[9];
  for (int col = 0; col < 3; ++col) {
    double e[3] = {0.0, 0.0, 0.0}, y[3];
    e[col] = 1.0;
    w_apply(phi, a, b, c, e, y);
    for (int r = 0; r < 3; ++r) Wm[3 * r + col] = y[r];
  }
  const double A00 = Wm[4] * Wm[8] - Wm[5] * Wm[7], A01 = Wm[2] * Wm[7] - Wm[1] * Wm[8],
               A02 = Wm[1] * Wm[5] - Wm[2] * Wm[4];
  const double A10 = Wm[5] * Wm[6] - Wm[3] * Wm[8], A11 = Wm[0] * Wm[8] - Wm[2] * Wm[6],
               A12 = Wm[2] * Wm[3] - Wm[0] * Wm[5];
  const double A20 = Wm[3] * Wm[7] - Wm[4] * Wm[6], A21 = Wm[1] * Wm[6] - Wm[0] * Wm[7],
               A22 = Wm[0] * Wm[4] - Wm[1] * Wm[3];
  const double det = Wm[0] * A00 + Wm[1] * A10 + Wm[2] * A20;
  const double* t = S.t;
  xi[0] = (A00 * t[0] + A01 * t[1] + A02 * t[2]) / det;
  xi[1] = (A10 * t[0] + A11 * t[1] + A12 * t[2]) / det;
  xi[2] = (A20 * t[0] + A21 * t[1] + A22 * t[2]) / det;
}

// Eq. 5 (smoothness, loop = 0): log(dS^-1 Sa^-1 Sb); Eq. 6 (loop = 1): log(dS Sa^-1 Sb)
void pgo_residual(const Sim3& dS, const Sim3& Sa, const Sim3& Sb, int loop, double r[7]) {
  const Sim3 rel = sim3_mul(sim3_inv(Sa), Sb);
  sim3_log(sim3_mul(loop ? dS : sim3_inv(dS), rel), r);
}

struct PgoProblem {
  int N, F;
  std::vector<Sim3> S, dS;
  std::vector<int> fa, fb, loop;
};

double pgo_cost(const PgoProblem& P, const std::vector<Sim3>& S) {
  double c = 0.0, r[7];
  for (int f = 0; f < P.F; ++f) {
    pgo_residual(P.dS[f], S[P.fa[f]], S[P.fb[f]], P.loop[f], r);
    for (double v : r) c += v * v;
  }
  return c;
}

}  // namespace

extern "C" {

void oracle_sim3_exp(const double* xi, double* out) { sim3_store(sim3_exp(xi), out); }

void oracle_sim3_log(const double* S, double* xi) { sim3_log(sim3_load(S), xi); }

// residuals [F,7] of the factors at the given similarities
void oracle_pgo_residuals(int N, int F, const double* S, const double* dS, const int* fa, const int* fb,
                          const int* loop, double* r) {
  for (int f = 0; f < F; ++f)
    pgo_residual(sim3_load(dS + 8 * (size_t)f), sim3_load(S + 8 * (size_t)fa[f]), sim3_load(S + 8 * (size_t)fb[f]),
                 loop[f], r + 7 * (size_t)f);
}

// Levenberg-Marquardt on Eq. 7 (Sec. 3.3): S_0 held (gauge), S_i <- S_i Exp(d_i)
// for i >= 1; Jacobians by central differences (step h) of each factor's
// residual in the 7 coordinates of each of its two similarities; normal
// equations H = J^T J, g = J^T r; step from (H + lambda diag(H)) d = -g;
// accepted (lambda /= 10) if it lowers the cost, else rejected (lambda *= 10).
// S [N,8] in place; cost [iters+1] (the cost before each iteration and at the
// end), accepted [iters].  Returns 4 if a system is not positive definite.
int oracle_pgo_lm(int N, int F, double* S, const double* dS, const int* fa, const int* fb, const int* loop,
                  int iters, double lambda0, double h, double* cost, int* accepted) {
  for (int f = 0; f < F; ++f)
    if (fa[f] < 0 || fa[f] >= N || fb[f] < 0 || fb[f] >= N) return 1;
  PgoProblem P;
  P.N = N;
  P.F = F;
  for (int i = 0; i < N; ++i) P.S.push_back(sim3_load(S + 8 * (size_t)i));
  for (int f = 0; f < F; ++f) {
    P.dS.push_back(sim3_load(dS + 8 * (size_t)f));
    P.fa.push_back(fa[f]);
    P.fb.push_back(fb[f]);
    P.loop.push_back(loop[f]);
  }
  const int n = 7 * (N - 1);
  double lambda = lambda0;
  double cur = pgo_cost(P, P.S);
  for (int it = 0; it < iters; ++it) {
    cost[it] = cur;
    std::vector<double> H((size_t)n * n, 0.0), g(n, 0.0);
    for (int f = 0; f < F; ++f) {
      const int ab[2] = {P.fa[f], P.fb[f]};
      double r[7], J[2][7][7];  // J[side][residual row][coordinate]
      pgo_residual(P.dS[f], P.S[ab[0]], P.S[ab[1]], P.loop[f], r);
      for (int side = 0; side < 2; ++side)
        for (int m = 0; m < 7; ++m) {
          double d[7] = {0, 0, 0, 0, 0, 0, 0}, rp[7], rm[7];
          d[m] = h;
          Sim3 Sp = sim3_mul(P.S[ab[side]], sim3_exp(d));
          d[m] = -h;
          Sim3 Sm = sim3_mul(P.S[ab[side]], sim3_exp(d));
          pgo_residual(P.dS[f], side == 0 ? Sp : P.S[ab[0]], side == 1 ? Sp : P.S[ab[1]], P.loop[f], rp);
          pgo_residual(P.dS[f], side == 0 ? Sm : P.S[ab[0]], side == 1 ? Sm : P.S[ab[1]], P.loop[f], rm);
          for (int row = 0; row < 7; ++row) J[side][row][m] = (rp[row] - rm[row]) / (2.0 * h);
        }
      for (int sa = 0; sa < 2; ++sa) {
        if (ab[sa] == 0) continue;
        const int oa = 7 * (ab[sa] - 1);
        for (int m = 0; m < 7; ++m) {
          double gm = 0.0;
          for (int row = 0; row < 7; ++row) gm += J[sa][row][m] * r[row];
          g[oa + m] += gm;
        }
        for (int sb = 0; sb < 2; ++sb) {
          if (ab[sb] == 0) continue;
          const int ob = 7 * (ab[sb] - 1);
          for (int m = 0; m < 7; ++m)
            for (int k = 0; k < 7; ++k) {
              double hv = 0.0;
              for (int row = 0; row < 7; ++row) hv += J[sa][row][m] * J[sb][row][k];
              H[(size_t)(oa + m) * n + ob + k] += hv;
            }
        }
      }
    }
    for (int i = 0; i < n; ++i) H[(size_t)i * n + i] *= 1.0 + lambda;
    std::vector<double> rhs(n), d;
    for (int i = 0; i < n; ++i) rhs[i] = -g[i];
    if (cholesky_solve(H, n, rhs, d)) return 4;
    std::vector<Sim3> cand = P.S;
    for (int i = 1; i < N; ++i) cand[i] = sim3_mul(P.S[i], sim3_exp(&d[7 * (i - 1)]));
    const double c = pgo_cost(P, cand);
    if (c < cur) {
      P.S = cand;
      cur = c;
      lambda /= 10.0;
      accepted[it] = 1;
    } else {
      lambda *= 10.0;
      accepted[it] = 0;
    }
  }
  cost[iters] = cur;
  for (int i = 0; i < N; ++i) sim3_store(P.S[i], S + 8 * (size_t)i);
  return 0;
}

}  // extern "C"
