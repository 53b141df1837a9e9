// Sim(3) pose-graph optimisation (Sec. 3.3 "Optimization", Eqs. 5-7):
// Levenberg-Marquardt over N similarities with the first one held, smoothness
// factors log(dS^-1 Sa^-1 Sb) (Eq. 5) and loop factors log(dS Sa^-1 Sb)
// (Eq. 6), the sum of their squares being Eq. 7.
//
// Every iteration runs on the device with no host round trip:
//   k_pgo_lin     one warp per factor: the residual and its 7x14 Jacobian by
//                 central differences in the right-perturbation coordinates
//                 S <- S Exp(d) of both similarities (lanes 0-27 one probe
//                 each, lane 28 the residual), then J^T J and -J^T r
//                 accumulated into the tiled FP64 lower triangle and the
//                 right-hand side of the library's dense pose system;
//   k_pgo_damp    H + lambda diag(H), identity on the padding;
//   dpv_solve     the library's pose solver (one-CTA LDL^T for 7(N-1) <= 256,
//                 the tiled tcgen05 factorisation with FP64 refinement above);
//   k_pgo_cand    candidate S_i Exp(dx_i);
//   k_pgo_cost    squared residual of each factor at the candidate;
//   k_pgo_decide  one CTA: the cost summed in a fixed order (deterministic),
//                 then the LM decision (accept and lambda / 10, or reject and
//                 lambda * 10), recorded in the cost and acceptance arrays;
//   k_pgo_commit  the candidate copied over S where it was accepted.
// A similarity is stored as (tx, ty, tz, qx, qy, qz, qw, s) and maps x to
// s R(q) x + t; its tangent vector is (rho, phi, sigma).
#include <cmath>

#include "internal.cuh"

namespace {

constexpr int PG_WARPS = 4;   // factors per CTA of k_pgo_lin
constexpr int PG_RED = 1024;  // threads of k_pgo_decide

struct Sim {
  double t[3], q[4], s;
};

__device__ __forceinline__ Sim pg_load(const double* __restrict__ v) {
  Sim S;
  S.t[0] = v[0]; S.t[1] = v[1]; S.t[2] = v[2];
  S.q[0] = v[3]; S.q[1] = v[4]; S.q[2] = v[5]; S.q[3] = v[6];
  S.s = v[7];
  return S;
}

__device__ __forceinline__ void pg_store(const Sim& S, double* __restrict__ v) {
  v[0] = S.t[0]; v[1] = S.t[1]; v[2] = S.t[2];
  v[3] = S.q[0]; v[4] = S.q[1]; v[5] = S.q[2]; v[6] = S.q[3];
  v[7] = S.s;
}

// y = R(q) x, through the quaternion sandwich: y = x + 2w (v x x) + 2 v x (v x x)
__device__ __forceinline__ void pg_rotate(const double* q, const double* x, double* y) {
  const double c0 = q[1] * x[2] - q[2] * x[1], c1 = q[2] * x[0] - q[0] * x[2], c2 = q[0] * x[1] - q[1] * x[0];
  const double d0 = q[1] * c2 - q[2] * c1, d1 = q[2] * c0 - q[0] * c2, d2 = q[0] * c1 - q[1] * c0;
  y[0] = x[0] + 2.0 * (q[3] * c0 + d0);
  y[1] = x[1] + 2.0 * (q[3] * c1 + d1);
  y[2] = x[2] + 2.0 * (q[3] * c2 + d2);
}

// A B (apply B, then A)
__device__ __forceinline__ Sim pg_mul(const Sim& A, const Sim& B) {
  Sim C;
  const double* a = A.q;
  const double* b = B.q;
  C.q[0] = a[3] * b[0] + a[0] * b[3] + a[1] * b[2] - a[2] * b[1];
  C.q[1] = a[3] * b[1] - a[0] * b[2] + a[1] * b[3] + a[2] * b[0];
  C.q[2] = a[3] * b[2] + a[0] * b[1] - a[1] * b[0] + a[2] * b[3];
  C.q[3] = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
  double r[3];
  pg_rotate(A.q, B.t, r);
  for (int k = 0; k < 3; ++k) C.t[k] = A.s * r[k] + A.t[k];
  C.s = A.s * B.s;
  return C;
}

__device__ __forceinline__ Sim pg_inv(const Sim& A) {
  Sim B;
  B.q[0] = -A.q[0]; B.q[1] = -A.q[1]; B.q[2] = -A.q[2]; B.q[3] = A.q[3];
  double r[3];
  pg_rotate(B.q, A.t, r);
  const double is = 1.0 / A.s;
  for (int k = 0; k < 3; ++k) B.t[k] = -is * r[k];
  B.s = is;
  return B;
}

// The map rho -> t of Exp is W = integral over tau in [0, 1] of
// exp(tau ([phi]x + sigma I)) = a I + b [phi]x + c [phi]x^2 with
//   a = m0,  b = sum_j (-1)^j th^2j m_{2j+1} / (2j+1)!,
//   c = sum_j (-1)^j th^2j m_{2j+2} / (2j+2)!,  m_k = int tau^k e^{sigma tau}.
// Near th = 0 the first two terms of each series (th < 1e-4: the next terms
// are below 1e-17 relative); above, the closed forms of the two integrals.
__device__ void pg_moments(double sg, double* m) {  // m[0..4]
  if (fabs(sg) < 2.0) {
    double tj = 1.0;  // sigma^j / j!
    for (int k = 0; k < 5; ++k) m[k] = 0.0;
    for (int j = 0; j < 40; ++j) {
#pragma unroll
      for (int k = 0; k < 5; ++k) m[k] += tj / (double)(k + j + 1);
      tj *= sg / (double)(j + 1);
      if (fabs(tj) < 1e-18) break;
    }
    return;
  }
  const double e = exp(sg);
  m[0] = expm1(sg) / sg;
  for (int k = 1; k < 5; ++k) m[k] = (e - k * m[k - 1]) / sg;
}

__device__ __forceinline__ void pg_wcoef(double th, double sg, double& a, double& b, double& c) {
  if (th < 1e-4) {
    double m[5];
    pg_moments(sg, m);
    const double t2 = th * th;
    a = m[0];
    b = m[1] - t2 * m[3] / 6.0;
    c = 0.5 * m[2] - t2 * m[4] / 24.0;
    return;
  }
  a = sg == 0.0 ? 1.0 : expm1(sg) / sg;
  double sn, cs;
  sincos(th, &sn, &cs);
  const double e = exp(sg), den = sg * sg + th * th;
  b = (e * (sg * sn - th * cs) + th) / (th * den);
  c = (a - (e * (sg * cs + th * sn) - sg) / den) / (th * th);
}

// y = (a I + b [phi]x + c [phi]x^2) x
__device__ __forceinline__ void pg_wmul(const double* p, double a, double b, double c, const double* x, double* y) {
  const double u0 = p[1] * x[2] - p[2] * x[1], u1 = p[2] * x[0] - p[0] * x[2], u2 = p[0] * x[1] - p[1] * x[0];
  const double w0 = p[1] * u2 - p[2] * u1, w1 = p[2] * u0 - p[0] * u2, w2 = p[0] * u1 - p[1] * u0;
  y[0] = a * x[0] + b * u0 + c * w0;
  y[1] = a * x[1] + b * u1 + c * w1;
  y[2] = a * x[2] + b * u2 + c * w2;
}

__device__ Sim pg_exp(const double* xi) {
  const double* rho = xi;
  const double* phi = xi + 3;
  const double sg = xi[6];
  const double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
  Sim S;
  double hs, hc;  // sin(th/2)/th, cos(th/2)
  if (th < 1e-4) {
    const double t2 = th * th;
    hs = 0.5 - t2 / 48.0;
    hc = 1.0 - t2 / 8.0;
  } else {
    double sn;
    sincos(0.5 * th, &sn, &hc);
    hs = sn / th;
  }
  S.q[0] = hs * phi[0]; S.q[1] = hs * phi[1]; S.q[2] = hs * phi[2]; S.q[3] = hc;
  double a, b, c;
  pg_wcoef(th, sg, a, b, c);
  pg_wmul(phi, a, b, c, rho, S.t);
  S.s = exp(sg);
  return S;
}

__device__ void pg_log(const Sim& S, double* xi) {
  const double sgn = S.q[3] < 0.0 ? -1.0 : 1.0;  // q and -q are the same rotation
  const double v0 = sgn * S.q[0], v1 = sgn * S.q[1], v2 = sgn * S.q[2], w = sgn * S.q[3];
  const double vn = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
  const double th = 2.0 * atan2(vn, w);
  // th / |v|, by its series 2/w (1 - v^2 / (3 w^2)) where |v| is tiny
  const double f = vn < 1e-8 ? 2.0 / w * (1.0 - vn * vn / (3.0 * w * w)) : th / vn;
  double* phi = xi + 3;
  phi[0] = f * v0; phi[1] = f * v1; phi[2] = f * v2;
  const double sg = log(S.s);
  xi[6] = sg;
  double a, b, c;
  pg_wcoef(th, sg, a, b, c);
  // rho = W^-1 t by Cramer's rule on the columns of W
  double c0[3], c1[3], c2[3];
  const double e0[3] = {1.0, 0.0, 0.0}, e1[3] = {0.0, 1.0, 0.0}, e2[3] = {0.0, 0.0, 1.0};
  pg_wmul(phi, a, b, c, e0, c0);
  pg_wmul(phi, a, b, c, e1, c1);
  pg_wmul(phi, a, b, c, e2, c2);
  // rows of the adjugate are the cross products of column pairs
  const double x0[3] = {c1[1] * c2[2] - c1[2] * c2[1], c1[2] * c2[0] - c1[0] * c2[2], c1[0] * c2[1] - c1[1] * c2[0]};
  const double x1[3] = {c2[1] * c0[2] - c2[2] * c0[1], c2[2] * c0[0] - c2[0] * c0[2], c2[0] * c0[1] - c2[1] * c0[0]};
  const double x2[3] = {c0[1] * c1[2] - c0[2] * c1[1], c0[2] * c1[0] - c0[0] * c1[2], c0[0] * c1[1] - c0[1] * c1[0]};
  const double idet = 1.0 / (c0[0] * x0[0] + c0[1] * x0[1] + c0[2] * x0[2]);
  const double* t = S.t;
  xi[0] = idet * (x0[0] * t[0] + x0[1] * t[1] + x0[2] * t[2]);
  xi[1] = idet * (x1[0] * t[0] + x1[1] * t[1] + x1[2] * t[2]);
  xi[2] = idet * (x2[0] * t[0] + x2[1] * t[1] + x2[2] * t[2]);
}

// the factor's measurement on the left: dS^-1 (Eq. 5) or dS (Eq. 6)
__device__ __forceinline__ void pg_residual(const Sim& L, const Sim& Sa, const Sim& Sb, double* r) {
  pg_log(pg_mul(L, pg_mul(pg_inv(Sa), Sb)), r);
}

__device__ __forceinline__ Sim pg_left(const double* dS, int loop) {
  const Sim m = pg_load(dS);
  return loop ? m : pg_inv(m);
}

// Exp of x times the m-th tangent axis (the central-difference probes):
// rho_m gives the translation x e_m exactly; phi_m the rotation by x about
// axis m (sin(x/2), cos(x/2) by their series, |x| << 1e-4); sigma the scale
// e^x.  Exp(-x e_m) is the inverse of Exp(x e_m).
__device__ __forceinline__ Sim pg_exp_axis(int m, double x) {
  Sim E;
  E.t[0] = E.t[1] = E.t[2] = 0.0;
  E.q[0] = E.q[1] = E.q[2] = 0.0;
  E.q[3] = 1.0;
  E.s = 1.0;
  if (m < 3) {
    E.t[m] = x;
  } else if (m < 6) {
    const double x2 = x * x;
    E.q[m - 3] = x * (0.5 - x2 / 48.0);
    E.q[3] = 1.0 - x2 / 8.0;
  } else {
    E.s = exp(x);
  }
  return E;
}

__global__ void __launch_bounds__(32 * PG_WARPS) k_pgo_lin(int N, int F, const double* __restrict__ S,
                                                             const double* __restrict__ dS,
                                                             const int* __restrict__ fa, const int* __restrict__ fb,
                                                             const int* __restrict__ loop, double h, double* Sys,
                                                             int TS, double* y, int* status) {
  // residuals of the 28 probes (column c = l / 2 of J, sign + for even l),
  // then the unperturbed one; then the columns of J and the residual
  __shared__ double Rsh[PG_WARPS][29][8];
  __shared__ double Jsh[PG_WARPS][15][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double (*R)[8] = Rsh[wid];
  double (*J)[8] = Jsh[wid];
  for (int f = blockIdx.x * PG_WARPS + wid; f < F; f += gridDim.x * PG_WARPS) {
    const int a = fa[f], b = fb[f];
    if (a < 0 || a >= N || b < 0 || b >= N || a == b) {
      if (lane == 0) dpv_set_status(status, DST_BAD_INDEX);
      continue;
    }
    if (lane < 29) {
      // r = log(L Sa^-1 Sb) with L = dS^-1 (Eq. 5) or dS (Eq. 6); with
      // M = Sa^-1 Sb the probes are log(L M E) for Sb <- Sb E and
      // log(L E^-1 M) for Sa <- Sa E
      const Sim L = pg_left(dS + 8 * (size_t)f, loop[f]);
      const Sim M = pg_mul(pg_inv(pg_load(S + 8 * (size_t)a)), pg_load(S + 8 * (size_t)b));
      double r[7];
      if (lane == 28) {
        pg_log(pg_mul(L, M), r);
      } else {
        const int c = lane >> 1, side = c / 7, m = c - 7 * side;
        const double x = (lane & 1) ? -h : h;
        if (side) pg_log(pg_mul(L, pg_mul(M, pg_exp_axis(m, x))), r);
        else pg_log(pg_mul(L, pg_mul(pg_exp_axis(m, -x), M)), r);
      }
#pragma unroll
      for (int k = 0; k < 7; ++k) R[lane][k] = r[k];
    }
    __syncwarp();
    if (lane < 15) {
      const double ih = 0.5 / h;
#pragma unroll
      for (int k = 0; k < 7; ++k) J[lane][k] = lane == 14 ? R[28][k] : (R[2 * lane][k] - R[2 * lane + 1][k]) * ih;
    }
    __syncwarp();
    // unknowns: frame i >= 1 at 7 (i - 1); frame 0 is held
    const int oa = 7 * (a - 1), ob = 7 * (b - 1);
    if (lane < 14) {
      const int side = lane / 7, m = lane - 7 * side;
      const int o = side ? ob : oa;
      if (o >= 0) {
        double g = 0.0;
#pragma unroll
        for (int k = 0; k < 7; ++k) g += J[lane][k] * J[14][k];
        dpv_red_add(y + o + m, -g);
      }
    }
    for (int e = lane; e < 196; e += 32) {
      const int u = e / 14, v = e - 14 * (e / 14);
      const int ou = u < 7 ? oa : ob, ov = v < 7 ? oa : ob;
      if (ou < 0 || ov < 0) continue;
      const int Rr = ou + (u < 7 ? u : u - 7), Cc = ov + (v < 7 ? v : v - 7);
      if (Rr < Cc) continue;  // lower triangle only
      double hv = 0.0;
#pragma unroll
      for (int k = 0; k < 7; ++k) hv += J[u][k] * J[v][k];
      dpv_red_add(Sys + dpv_s_index(Rr, Cc, TS), hv);
    }
    __syncwarp();
  }
}

// H + lambda diag(H) on the unknowns, 1 on the padding diagonal
__global__ void k_pgo_damp(int n, int n_pad, int TS, double* Sys, const double* __restrict__ lm) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_pad) return;
  double* d = Sys + dpv_s_index(r, r, TS);
  *d = r < n ? *d * (1.0 + lm[0]) : 1.0;
}

__global__ void k_pgo_cand(int N, const double* __restrict__ S, const double* __restrict__ dx, double* cand) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (i == 0) {
    for (int k = 0; k < 8; ++k) cand[k] = S[k];
    return;
  }
  double d[7];
  for (int k = 0; k < 7; ++k) d[k] = dx[7 * (i - 1) + k];
  pg_store(pg_mul(pg_load(S + 8 * (size_t)i), pg_exp(d)), cand + 8 * (size_t)i);
}

__global__ void k_pgo_cost(int N, int F, const double* __restrict__ S, const double* __restrict__ dS,
                           const int* __restrict__ fa, const int* __restrict__ fb, const int* __restrict__ loop,
                           double* fcost) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int a = fa[f], b = fb[f];
  if (a < 0 || a >= N || b < 0 || b >= N || a == b) {
    fcost[f] = 0.0;  // flagged by k_pgo_lin
    return;
  }
  double r[7];
  pg_residual(pg_left(dS + 8 * (size_t)f, loop[f]), pg_load(S + 8 * (size_t)a), pg_load(S + 8 * (size_t)b), r);
  double c = 0.0;
  for (int k = 0; k < 7; ++k) c += r[k] * r[k];
  fcost[f] = c;
}

// lm = (lambda, current cost, accepted flag).  it < 0: the initial cost.
__global__ void __launch_bounds__(PG_RED) k_pgo_decide(int F, const double* __restrict__ fcost, double* lm, int it,
                                                      double* cost, int* accepted) {
  __shared__ double part[PG_RED];
  double s = 0.0;
  for (int f = threadIdx.x; f < F; f += PG_RED) s += fcost[f];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = PG_RED / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double c = part[0];
  if (it < 0) {
    lm[1] = c;
    lm[2] = 0.0;
    cost[0] = c;
    return;
  }
  const int acc = c < lm[1];
  if (acc) {
    lm[1] = c;
    lm[0] *= 0.1;
  } else {
    lm[0] *= 10.0;
  }
  lm[2] = acc;
  cost[it + 1] = lm[1];
  if (accepted) accepted[it] = acc;
}

__global__ void k_pgo_commit(int N, double* S, const double* __restrict__ cand, const double* __restrict__ lm) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8 * N || lm[2] == 0.0) return;
  S[e] = cand[e];
}

__global__ void k_pgo_init(double* lm, double lambda0) {
  lm[0] = lambda0;
  lm[1] = 0.0;
  lm[2] = 0.0;
}

}  // namespace

extern "C" ba_status_t ba_pgo_lm(ba_handle_t h, int N, int F, double* S, const double* dS, const int* fa,
                                 const int* fb, const int* loop, int iters, double lambda0, double fd_step,
                                 double* cost, int* accepted) {
  if (!h) return BA_ERR_INVALID_ARG;
  if (N < 1 || F < 0 || iters < 0 || N > BA_PGO_MAX_FRAMES || !(lambda0 > 0.0) || !(fd_step > 0.0) ||
      !(fd_step < 1e-2))
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_pgo_lm: sizes or parameters out of range");
  if (!S || !cost || (F > 0 && (!dS || !fa || !fb || !loop)))
    return dpv_fail(h, BA_ERR_INVALID_ARG, "ba_pgo_lm: null pointer");
  const int n = 7 * (N - 1);
  ba_status_t s;
  if ((s = dpv_ensure_generic_system(h, n))) return s;
  Workspace* ws = h->ws;
  if ((s = dpv_grow(h, ws->pgo, 3 + 8LL * N + (F > 0 ? F : 1), "pose-graph scratch"))) return s;
  double* lm = ws->pgo.p;
  double* cand = lm + 3;
  double* fcost = cand + 8LL * N;
  const SysDesc& d = h->sys[0];
  cudaStream_t st = h->stream;
  dpv_prof_begin(h, BA_KERNEL_PGO);
  k_pgo_init<<<1, 1, 0, st>>>(lm, lambda0);
  if (F > 0) k_pgo_cost<<<(F + 127) / 128, 128, 0, st>>>(N, F, S, dS, fa, fb, loop, fcost);
  else DPV_CUDA(h, cudaMemsetAsync(fcost, 0, sizeof(double), st));
  k_pgo_decide<<<1, PG_RED, 0, st>>>(F, fcost, lm, -1, cost, accepted);
  h->launches += F > 0 ? 3 : 2;
  dpv_prof_end(h);
  DPV_CUDA(h, cudaGetLastError());
  const int lin_blocks = std::max(1, std::min((F + PG_WARPS - 1) / PG_WARPS, 16 * h->num_sms));
  for (int it = 0; it < iters && n > 0; ++it) {
    dpv_prof_begin(h, BA_KERNEL_PGO);
    DPV_CUDA(h, cudaMemsetAsync(ws->S.p, 0, sizeof(double) * h->nS, st));
    DPV_CUDA(h, cudaMemsetAsync(ws->y.p, 0, sizeof(double) * h->n_pad, st));
    if (F > 0)
      k_pgo_lin<<<lin_blocks, 32 * PG_WARPS, 0, st>>>(N, F, S, dS, fa, fb, loop, fd_step, ws->S.p + d.soff, d.TS,
                                                     ws->y.p + d.voff, ws->status);
    k_pgo_damp<<<(d.n_pad + 255) / 256, 256, 0, st>>>(n, d.n_pad, d.TS, ws->S.p + d.soff, lm);
    h->launches += F > 0 ? 2 : 1;
    dpv_prof_end(h);
    DPV_CUDA(h, cudaGetLastError());
    // (the solver records its own kernel classes)
    int retracted = 0;
    dpv_prof_begin(h, BA_KERNEL_SOLVE);
    s = dpv_solve(h, &retracted, 0);
    dpv_prof_end(h);
    if (s) return s;
    dpv_prof_begin(h, BA_KERNEL_PGO);
    k_pgo_cand<<<(N + 127) / 128, 128, 0, st>>>(N, S, ws->dx.p + d.voff, cand);
    if (F > 0) k_pgo_cost<<<(F + 127) / 128, 128, 0, st>>>(N, F, cand, dS, fa, fb, loop, fcost);
    k_pgo_decide<<<1, PG_RED, 0, st>>>(F, fcost, lm, it, cost, accepted);
    k_pgo_commit<<<(8 * N + 255) / 256, 256, 0, st>>>(N, S, cand, lm);
    h->launches += F > 0 ? 4 : 3;
    dpv_prof_end(h);
    DPV_CUDA(h, cudaGetLastError());
  }
  // no unknowns (N = 1): nothing moves, every iteration records the cost
  for (int it = 0; it < iters && n == 0; ++it) {
    k_pgo_decide<<<1, PG_RED, 0, st>>>(F, fcost, lm, it, cost, accepted);
    ++h->launches;
  }
  DPV_CUDA(h, cudaGetLastError());
  return BA_OK;
}
