// Log-conformation Giesekus / Oldroyd-B update on coarse centres (Section 3.2.3).
//
// RH of Eq. NS41 with the relaxation acting toward Theta = 0:
//   RH = -div(u Theta) + (Omega Theta - Theta Omega) + 2 B
//        - e^{-Theta} [I + alpha (e^Theta - I)] (e^Theta - I)/lambda_H,
// (Giesekus mobility alpha; alpha = 0 is Oldroyd-B, (e^{-Theta} - I)/lambda_H),
// Omega and B from the decomposition of Eqs. NS21-NS24 with
// Theta = R diag(theta) R^T, lambda = e^theta, M~ = R^T (grad u)^T R.
// In the eigenbasis RH~ = R^T (RH + div(u Theta)) R is symmetric with
//   RH~_aa = 2 m_aa + [(e^{-theta_a} - 1) - alpha (e^{theta_a} - 1)(1 - e^{-theta_a})]/lambda_H,
//   RH~_ab = omega_ab (theta_b - theta_a)
//          = (lambda_b m_ab + lambda_a m_ba) (theta_b - theta_a)/(lambda_b - lambda_a),
// evaluated as (e^d m_ab + m_ba) d/expm1(d), d = theta_b - theta_a, which is
// finite as d -> 0 and equals there the equal-eigenvalue limit m_ab + m_ba
// (Omega = 0, B = sym(grad u^T), the zero-stress rule after Eq. NS24).
// RK2-TVD: Theta1 = Theta^n + dt RH(Theta^n) (Eq. NS42); Theta^{n+1} =
// Theta^n/2 + (Theta1 + dt RH(Theta1))/2 (Eq. NS44); tau_p = (mu_p/lambda_H)
// (R e^Lambda R^T - I) (Eq. NS46); the momentum equation receives
// tau = (1 + phi)/2 tau_p (Eq. NS12, droplet phase viscoelastic); in approach 1
// (Eq. NS11) lambda_H, mu_p and alpha are linear in the restricted phi at each
// centre and tau = tau_p.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "weno.cuh"

namespace pf {

template <class T>
__device__ __forceinline__ T dexpm1(T d);
template <>
__device__ __forceinline__ float dexpm1<float>(float d) {  // d / expm1(d)
  if (fabsf(d) < 1e-3f) return 1.f - 0.5f * d + d * d * (1.f / 12.f);
  return d / expm1f(d);
}
template <>
__device__ __forceinline__ double dexpm1<double>(double d) {
  if (fabs(d) < 1e-6) return 1.0 - 0.5 * d + d * d * (1.0 / 12.0);
  return d / expm1(d);
}

template <>
__device__ __forceinline__ Dual dexpm1<Dual>(Dual d) {
  if (fabs(d.v) < 1e-6) return 1.0 - 0.5 * d + d * d * (1.0 / 12.0);
  return d / expm1(d);
}

template <class T>
__device__ __forceinline__ T fexp(T x) { return exp(x); }

// x / (e^x - 1) for x <= 0 given ex = e^x (which the caller already has).
// FP32: for x > -1/4 the Bernoulli series 1 - x/2 + x^2/12 - x^4/720 +
// x^6/30240 - x^8/1209600 (next term below 3e-14 there); below, x/(ex - 1),
// where ex - 1 <= -0.22 carries no cancellation.  FP64 and Dual: dexpm1.
template <class T>
__device__ __forceinline__ T dexpm1_e(T x, T ex) {
  (void)ex;
  return dexpm1<T>(x);
}
template <>
__device__ __forceinline__ float dexpm1_e<float>(float x, float ex) {
  if (x > -0.25f) {
    const float x2 = x * x;
    float p = fmaf(x2, -1.f / 1209600.f, 1.f / 30240.f);
    p = fmaf(x2, p, -1.f / 720.f);
    p = fmaf(x2, p, 1.f / 12.f);
    return fmaf(x2, p, fmaf(x, -0.5f, 1.f));
  }
  return __fdividef(x, ex - 1.f);
}
template <>
__device__ __forceinline__ float fexp<float>(float x) { return __expf(x); }

// Symmetric N x N matrix held as its N diagonal and N(N-1)/2 off-diagonal
// entries; off-diagonal slot of (p, q): 2D (0,1) -> 0; 3D (0,1) -> 0,
// (0,2) -> 1, (1,2) -> 2.
template <int N>
__device__ __forceinline__ constexpr int off_slot(int p, int q) {
  return N == 2 ? 0 : (p + q - 1);
}

// One Jacobi rotation P (P_pp = P_qq = c, P_pq = s, P_qp = -s) that zeroes
// a_pq: A <- P^T A P on the unique entries only, V <- V P.
template <class T, int N>
__device__ __forceinline__ void jacobi_rot_sym(T (&dg)[N], T (&of)[N == 2 ? 1 : 3], T (&V)[N][N], int p, int q) {
  const int pq = off_slot<N>(p, q);
  const T apq = of[pq];
  if (apq == (T)0) return;
  const T th = (dg[q] - dg[p]) / (2 * apq);
  const T ath = fabs(th);
  // t = sgn(th)/(|th| + sqrt(th^2 + 1)), the smaller root; 1/(2 th) when th^2 would overflow
  T t = ath > (T)1e15 ? (T)0.5 / ath : (T)1 / (ath + sqrt(ath * ath + (T)1));
  if (th < 0) t = -t;
  const T c = rsqrt(t * t + (T)1), s = t * c;
  dg[p] -= t * apq;
  dg[q] += t * apq;
  of[pq] = 0;
  if (N == 3) {
    const int r = 3 - p - q;
    const int rp = off_slot<N>(r < p ? r : p, r < p ? p : r), rq = off_slot<N>(r < q ? r : q, r < q ? q : r);
    const T arp = of[rp], arq = of[rq];
    of[rp] = c * arp - s * arq;
    of[rq] = s * arp + c * arq;
  }
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const T vrp = V[r][p], vrq = V[r][q];
    V[r][p] = c * vrp - s * vrq;
    V[r][q] = s * vrp + c * vrq;
  }
}

// FP32: the same rotation with tan(phi) written as g / (|h| + sqrt(h^2 + g^2)) sgn(h),
// h = a_qq - a_pp, g = 2 a_pq (equal to the smaller root above), one fast divide
// and reciprocal square roots; the rotation stays orthogonal to rounding.
template <int N>
__device__ __forceinline__ void jacobi_rot_sym_f(float (&dg)[N], float (&of)[N == 2 ? 1 : 3], float (&V)[N][N], int p,
                                                 int q) {
  const int pq = off_slot<N>(p, q);
  const float apq = of[pq];
  if (apq == 0.f) return;
  const float h = dg[q] - dg[p], g = 2.f * apq;
  const float a = fmaf(h, h, g * g);  // > 0 (apq != 0)
  const float r = a * rsqrtf(a);      // sqrt(a) to a few ulp: t is the rotation's own, c and s follow it
  float t = __fdividef(g, fabsf(h) + r);
  if (h < 0.f) t = -t;
  const float c = rsqrtf(fmaf(t, t, 1.f)), s = t * c;
  dg[p] -= t * apq;
  dg[q] += t * apq;
  of[pq] = 0.f;
  if (N == 3) {
    const int r3 = 3 - p - q;
    const int rp = off_slot<N>(r3 < p ? r3 : p, r3 < p ? p : r3), rq = off_slot<N>(r3 < q ? r3 : q, r3 < q ? q : r3);
    const float arp = of[rp], arq = of[rq];
    of[rp] = c * arp - s * arq;
    of[rq] = s * arp + c * arq;
  }
#pragma unroll
  for (int rr = 0; rr < N; ++rr) {
    const float vrp = V[rr][p], vrq = V[rr][q];
    V[rr][p] = c * vrp - s * vrq;
    V[rr][q] = s * vrp + c * vrq;
  }
}

// Symmetric 3 x 3 eigen-decomposition A = V diag(w) V^T in closed form (FP32,
// FP64), V orthonormal to rounding.  The mean m = tr A / 3 is removed and the
// rest scaled by its largest entry s, B = (A - m I)/s.  Of the roots
//   2 p cos(psi + 2 pi k/3),  p^2 = tr(B^2)/6,  psi = acos(det(B/p)/2)/3
// of B's characteristic polynomial (the trigonometric solution of the cubic),
// only the one farthest from the other two is used: k = 0 for psi < pi/6,
// else k = 2.  Its gap to the others is at least sqrt(3) p, so its
// eigenvector, the largest cross product of two rows of B - w I, is well
// conditioned, and its eigenvalue is taken again as the Rayleigh quotient of
// that vector.  The other two pairs come from diagonalising B on the plane
// orthogonal to it (one exact rotation), so a near-double eigenvalue costs no
// accuracy.  On entry (dg, of) hold A, on exit dg the eigenvalues and V the
// eigenvectors in columns.
// FP32 forms of the closed form's few non-FMA steps (a fast divide, the
// hardware cosine): they touch only the isolated root, whose eigenvalue is then
// taken again as a Rayleigh quotient, and the rotation of the pair, which stays
// orthogonal by construction; FP64 keeps the exact functions.
template <class T>
__device__ __forceinline__ T e3_div(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float e3_div<float>(float a, float b) { return __fdividef(a, b); }
template <class T>
__device__ __forceinline__ T e3_cos(T x) { return cos(x); }
template <>
__device__ __forceinline__ float e3_cos<float>(float x) { return __cosf(x); }

template <class T>
__device__ __forceinline__ void eig_sym3_closed(T (&dg)[3], T (&of)[3], T (&V)[3][3]) {
  const T m = (dg[0] + dg[1] + dg[2]) * (T)(1.0 / 3.0);
  T b[3][3];
  b[0][0] = dg[0] - m, b[1][1] = dg[1] - m, b[2][2] = dg[2] - m;
  b[0][1] = b[1][0] = of[0], b[0][2] = b[2][0] = of[1], b[1][2] = b[2][1] = of[2];
  T sc = (T)0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = a; c < 3; ++c) sc = fmax(sc, fabs(b[a][c]));
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) V[a][c] = (a == c) ? (T)1 : (T)0;
  if (sc == (T)0) {  // A = m I
    dg[0] = dg[1] = dg[2] = m;
    return;
  }
  const T isc = e3_div<T>((T)1, sc);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) b[a][c] *= isc;
  const T p2 = (b[0][0] * b[0][0] + b[1][1] * b[1][1] + b[2][2] * b[2][2] +
                (T)2 * (b[0][1] * b[0][1] + b[0][2] * b[0][2] + b[1][2] * b[1][2])) * (T)(1.0 / 6.0);
  const T ip = rsqrt(p2), p = p2 * ip;
  const T det = b[0][0] * (b[1][1] * b[2][2] - b[1][2] * b[1][2]) - b[0][1] * (b[0][1] * b[2][2] - b[1][2] * b[0][2]) +
                b[0][2] * (b[0][1] * b[1][2] - b[1][1] * b[0][2]);
  T r = (T)0.5 * det * ip * ip * ip;
  r = fmin(fmax(r, (T)-1), (T)1);
  const T psi = acos(r) * (T)(1.0 / 3.0);
  const T lam = (T)2 * p * e3_cos<T>(psi < (T)(3.14159265358979323846 / 6.0) ? psi : psi + (T)(4.0 * 3.14159265358979323846 / 3.0));
  // eigenvector of lam: the largest cross product of two rows of B - lam I
  T r0[3] = {b[0][0] - lam, b[0][1], b[0][2]}, r1[3] = {b[0][1], b[1][1] - lam, b[1][2]},
    r2[3] = {b[0][2], b[1][2], b[2][2] - lam};
  auto cross = [](const T (&x)[3], const T (&y)[3], T (&z)[3]) {
    z[0] = x[1] * y[2] - x[2] * y[1];
    z[1] = x[2] * y[0] - x[0] * y[2];
    z[2] = x[0] * y[1] - x[1] * y[0];
  };
  T v[3], c1[3], c2[3];
  cross(r0, r1, v);
  cross(r0, r2, c1);
  cross(r1, r2, c2);
  T n0 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const T n1 = c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2];
  const T n2 = c2[0] * c2[0] + c2[1] * c2[1] + c2[2] * c2[2];
  if (n1 > n0) {
    v[0] = c1[0], v[1] = c1[1], v[2] = c1[2];
    n0 = n1;
  }
  if (n2 > n0) {
    v[0] = c2[0], v[1] = c2[1], v[2] = c2[2];
    n0 = n2;
  }
  const T iv = rsqrt(n0);
  v[0] *= iv, v[1] *= iv, v[2] *= iv;
  // orthonormal pair spanning the plane orthogonal to v
  const T ax = fabs(v[0]), ay = fabs(v[1]), az = fabs(v[2]);
  const bool ex = ax <= ay && ax <= az, ey = !ex && ay <= az;  // the axis least aligned with v
  T u[3], w[3];
  // u = v x e (e the unit vector of that axis)
  u[0] = ex ? (T)0 : (ey ? -v[2] : v[1]);
  u[1] = ex ? v[2] : (ey ? (T)0 : -v[0]);
  u[2] = ex ? -v[1] : (ey ? v[0] : (T)0);
  const T iu = rsqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  u[0] *= iu, u[1] *= iu, u[2] *= iu;
  cross(v, u, w);
  auto quad = [&](const T (&x)[3], const T (&y)[3]) {  // x^T B y
    T t = (T)0;
#pragma unroll
    for (int a = 0; a < 3; ++a) t += x[a] * (b[a][0] * y[0] + b[a][1] * y[1] + b[a][2] * y[2]);
    return t;
  };
  const T lv = quad(v, v), a11 = quad(u, u), a12 = quad(u, w), a22 = quad(w, w);
  // one rotation diagonalises the 2 x 2 block [[a11, a12], [a12, a22]]
  // t = tan of the rotation angle, g/(|h| + sqrt(h^2 + g^2)) sgn h (h = a22 - a11,
  // g = 2 a12), the smaller root, without overflow
  T cs = (T)1, sn = (T)0, t = (T)0;
  if (a12 != (T)0) {
    const T hh = a22 - a11, gg = (T)2 * a12;
    const T aa = hh * hh + gg * gg;
    t = e3_div<T>(gg, fabs(hh) + aa * rsqrt(aa));
    if (hh < (T)0) t = -t;
    cs = rsqrt(t * t + (T)1);
    sn = t * cs;
  }
  dg[0] = m + sc * lv;
  dg[1] = m + sc * (a11 - t * a12);
  dg[2] = m + sc * (a22 + t * a12);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    V[a][0] = v[a];
    V[a][1] = cs * u[a] - sn * w[a];
    V[a][2] = sn * u[a] + cs * w[a];
  }
}

// symmetric eigen-decomposition A = V diag(w) V^T: in closed form for a 3 x 3
// in FP32 or FP64, else by cyclic Jacobi rotations (2 x 2: one rotation; the
// derivative-carrying type); on entry (dg, of) hold A, on exit dg holds the
// eigenvalues w
template <class T, int N>
__device__ __forceinline__ void eig_sym(T (&dg)[N], T (&of)[N == 2 ? 1 : 3], T (&V)[N][N]) {
  if constexpr (N == 3 && !IsDual<T>::value) {
    eig_sym3_closed<T>(dg, of, V);
    return;
  }
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int b = 0; b < N; ++b) V[a][b] = (a == b) ? (T)1 : (T)0;
  auto rot = [&](int p, int q) {
    if constexpr (std::is_same<T, float>::value) jacobi_rot_sym_f<N>(dg, of, V, p, q);
    else jacobi_rot_sym<T, N>(dg, of, V, p, q);
  };
  if (N == 2) {  // one rotation diagonalises a 2 x 2 matrix
    rot(0, 1);
    return;
  }
  const T eps2 = sizeof(T) == 4 ? (T)1e-14 : (T)1e-30;
#pragma unroll 1
  for (int sweep = 0; sweep < (sizeof(T) == 4 ? 6 : 10); ++sweep) {
    T off = 0, dia = 0;
#pragma unroll
    for (int a = 0; a < N; ++a) dia += dg[a] * dg[a];
#pragma unroll
    for (int o = 0; o < (N == 2 ? 1 : 3); ++o) off += of[o] * of[o];
    if (off <= eps2 * dia || off == (T)0) break;
    rot(0, 1);
    rot(0, 2);
    rot(1, 2);
  }
}

template <class T>
struct PolyIn {
  const T *u, *v, *w;  // u^{n+1} (w with both wall faces)
  const T* phic;       // restricted phi^{n+1} at centres
  const T* th[6];      // Theta to take RH of (component-major)
  const T* base[6];    // Theta^n (stage 2 only)
  T* out[6];           // Theta1 (stage 1) or Theta^{n+1} (stage 2)
  T* tau[6];           // weighted tau^{n+1} (stage 2)
};

// component maps: 2D (x, z) comps xx, xz, zz; 3D xx, yy, zz, xy, xz, yz
template <int N>
__device__ __forceinline__ int comp_of(int a, int b) {
  if (N == 2) return (a == b) ? (a == 0 ? 0 : 2) : 1;
  if (a == b) return a;
  const int s = a + b;  // (0,1) -> 3, (0,2) -> 4, (1,2) -> 5
  return s == 1 ? 3 : (s == 2 ? 4 : 5);
}

// The local part of RH at one cell: R H R^T of Eq. NS41 (everything but the
// advection), from Theta's unique components th0 and the velocity gradient
// L[a][b] = du_a/dx_b.  Returns it per component in s_out, and Theta's
// eigenbasis R and eigenvalues dg.
template <class T, int N>
__device__ __forceinline__ void lcr_rhs_local(const T (&th0)[N == 2 ? 3 : 6], const T (&L)[N][N], const PhysT<T>& q,
                                              T (&s_out)[N == 2 ? 3 : 6], T (&R)[N][N], T (&dg)[N]) {
  T of[N == 2 ? 1 : 3];
#pragma unroll
  for (int a = 0; a < N; ++a) dg[a] = th0[comp_of<N>(a, a)];
  if (N == 2) of[0] = th0[comp_of<N>(0, 1)];
  else {
    of[0] = th0[comp_of<N>(0, 1)];
    of[1] = th0[comp_of<N>(0, 2)];
    of[2] = th0[comp_of<N>(1, 2)];
  }
  eig_sym<T, N>(dg, of, R);
  // M~ = R^T L R
  T LR[N][N], Mt[N][N];
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int b = 0; b < N; ++b) {
      T s = 0;
#pragma unroll
      for (int c = 0; c < N; ++c) s += L[a][c] * R[c][b];
      LR[a][b] = s;
    }
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int b = 0; b < N; ++b) {
      T s = 0;
#pragma unroll
      for (int c = 0; c < N; ++c) s += R[c][a] * LR[c][b];
      Mt[a][b] = s;
    }
  // RH in the eigenbasis
  T H[N][N];
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const T em = fexp<T>(-dg[a]);
    T relax = em - (T)1;  // Oldroyd-B: e^{-theta} - 1
    if (q.ag != (T)0) relax -= q.ag * (fexp<T>(dg[a]) - (T)1) * ((T)1 - em);  // Giesekus
    H[a][a] = 2 * Mt[a][a] + relax * q.ilh;
#pragma unroll
    for (int b = a + 1; b < N; ++b) {
      const T dd = dg[b] - dg[a];
      T o;
      const T x = dd > 0 ? -dd : dd;  // -|dd|
      const T ex = fexp<T>(x);
      const T wgt = dexpm1_e<T>(x, ex);
      if (dd > 0) o = (Mt[a][b] + ex * Mt[b][a]) * wgt;
      else o = (ex * Mt[a][b] + Mt[b][a]) * wgt;
      H[a][b] = o;
      H[b][a] = o;
    }
  }
  // back to the physical basis: R H R^T
  T HR[N][N];
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int b = 0; b < N; ++b) {
      T s = 0;
#pragma unroll
      for (int c = 0; c < N; ++c) s += H[a][c] * R[b][c];
      HR[a][b] = s;
    }
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int b = a; b < N; ++b) {
      T s = 0;
#pragma unroll
      for (int c = 0; c < N; ++c) s += R[a][c] * HR[c][b];
      s_out[comp_of<N>(a, b)] = s;
    }
}

// The polymer constants at a coarse centre with restricted phi `ph`: in
// approach 1 (Eq. NS11) lambda_H, mu_p and alpha are linear in phi, and the
// stress weight is 1; otherwise the droplet's constants, weight (1 + phi)/2
// (Eq. NS12).  Returns the constants with ilh, ag and wtau set, and the
// weight of tau_p in `wgt`.
template <class T>
__device__ __forceinline__ PhysT<T> poly_at(const PhysT<T>& q, T ph, T& wgt) {
  PhysT<T> qc = q;
  if (q.ap1) {
    const T a = (T)0.5 * ((T)1 + ph), b = (T)0.5 * ((T)1 - ph);
    const T lh = a * q.lh1 + b * q.lh2;
    qc.ilh = (T)1 / lh;
    qc.ag = a * q.ag + b * q.ag2;
    qc.wtau = (a * q.mp1 + b * q.mp2) * qc.ilh;
    wgt = qc.wtau;
  } else {
    wgt = (T)0.5 * ((T)1 + ph) * q.wtau;
  }
  return qc;
}

// tau = (1 + phi)/2 (mu_p/lambda_H) (W e^theta W^T - I) from Theta's unique
// components (Eqs. NS12, NS46; Eq. NS11 in approach 1), with a decomposition
// of its own
template <class T, int N>
__device__ __forceinline__ void lcr_tau(const T (&th)[N == 2 ? 3 : 6], T phic, const PhysT<T>& q,
                                        T (&tau)[N == 2 ? 3 : 6]) {
  T dg[N], of[N == 2 ? 1 : 3], R[N][N];
#pragma unroll
  for (int a = 0; a < N; ++a) dg[a] = th[comp_of<N>(a, a)];
  if (N == 2) of[0] = th[comp_of<N>(0, 1)];
  else {
    of[0] = th[comp_of<N>(0, 1)];
    of[1] = th[comp_of<N>(0, 2)];
    of[2] = th[comp_of<N>(1, 2)];
  }
  eig_sym<T, N>(dg, of, R);
  T ex[N];
#pragma unroll
  for (int c = 0; c < N; ++c) ex[c] = fexp<T>(dg[c]);
  T wgt;
  (void)poly_at<T>(q, phic, wgt);
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int b = a; b < N; ++b) {
      T s = 0;
#pragma unroll
      for (int c = 0; c < N; ++c) s += R[a][c] * ex[c] * R[b][c];
      tau[comp_of<N>(a, b)] = wgt * (s - (a == b ? (T)1 : (T)0));
    }
}

// one RK2-TVD stage at one coarse cell; STAGE 2 also forms tau
template <class T, int N, int STAGE>
__device__ __forceinline__ void polymer_cell(const PolyIn<T>& P, const Dims& d, const PhysT<T>& q, const RowIdx& x) {
  const int nx = d.nx, plane = d.nx * d.ny;
  const T iD = q.iD;
  constexpr int NC = N == 2 ? 3 : 6;
  const int i = x.i, j = x.j, k = x.k;
  const int id = x.row * nx + i;
  // wrapped neighbour offsets, computed once
  const int ox = (i + 1 == nx) ? 1 - nx : 1, oxm = (i == 0) ? nx - 1 : -1;
  const int oy = N == 3 ? ((j + 1 == d.ny) ? (1 - d.ny) * nx : nx) : 0;
  const int oym = N == 3 ? ((j == 0) ? (d.ny - 1) * nx : -nx) : 0;
  const bool top = k + 1 == d.nz, bot = k == 0;
  const T* __restrict__ U = P.u;
  const T* __restrict__ Vv = P.v;
  const T* __restrict__ W = P.w;
  auto uc = [&](int c) -> T { return (T)0.5 * (U[c] + U[c + ox]); };
  auto wc = [&](int c) -> T { return (T)0.5 * (W[c] + W[c + plane]); };
  // velocity gradient L[a][b] = du_a/dx_b; wall ghosts 2 u_w - u_0 (tangential), w = 0
  T L[N][N];
  const T uc0 = uc(id);
  const T ucp = top ? q.uw2_top - uc0 : uc(id + plane);
  const T ucm = bot ? q.uw2_bot - uc0 : uc(id - plane);
  const T dudx = (U[id + ox] - U[id]) * iD;
  const T dudz = (ucp - ucm) * (T)0.5 * iD;
  const T dwdx = (wc(id + ox) - wc(id + oxm)) * (T)0.5 * iD;
  const T dwdz = (W[id + plane] - W[id]) * iD;
  if (N == 2) {
    L[0][0] = dudx;
    L[0][N - 1] = dudz;
    L[N - 1][0] = dwdx;
    L[N - 1][N - 1] = dwdz;
  } else {
    auto vc = [&](int c) -> T { return (T)0.5 * (Vv[c] + Vv[c + oy]); };
    const T vc0 = vc(id);
    const T vcp = top ? -vc0 : vc(id + plane);
    const T vcm = bot ? -vc0 : vc(id - plane);
    L[0][0] = dudx;
    L[0][1] = (uc(id + oy) - uc(id + oym)) * (T)0.5 * iD;
    L[0][N - 1] = dudz;
    L[1][0] = (vc(id + ox) - vc(id + oxm)) * (T)0.5 * iD;
    L[1][1] = (Vv[id + oy] - Vv[id]) * iD;
    L[1][N - 1] = (vcp - vcm) * (T)0.5 * iD;
    L[N - 1][0] = dwdx;
    L[N - 1][1] = (wc(id + oy) - wc(id + oym)) * (T)0.5 * iD;
    L[N - 1][N - 1] = dwdz;
  }
  // advection div(u Theta), conservative, no wall flux: WENO5-Z face values
  // (the paper's scheme) when selected, else central
  T adv[NC], th0[NC];
  if (q.weno) {
#pragma unroll
    for (int cq = 0; cq < NC; ++cq) {
      adv[cq] = weno_div_coarse<T>(P.th[cq], U, Vv, W, i, j, k, d, iD);
      th0[cq] = P.th[cq][id];
    }
  } else {
    const T ul = U[id], ur = U[id + ox];
    const T wb = W[id], wt = W[id + plane];
    const T vl = N == 3 ? Vv[id] : (T)0, vr = N == 3 ? Vv[id + oy] : (T)0;
#pragma unroll
    for (int cq = 0; cq < NC; ++cq) {
      const T* __restrict__ th = P.th[cq];
      const T t0 = th[id];
      T a = ur * (t0 + th[id + ox]) - ul * (th[id + oxm] + t0);
      if (!top) a += wt * (t0 + th[id + plane]);
      if (!bot) a -= wb * (th[id - plane] + t0);
      if (N == 3) a += vr * (t0 + th[id + oy]) - vl * (th[id + oym] + t0);
      adv[cq] = (T)0.5 * iD * a;
      th0[cq] = t0;
    }
  }
  // polymer constants of this centre (Eq. NS11 in approach 1)
  T wgt = (T)0;
  const PhysT<T> qc = q.ap1 ? poly_at<T>(q, P.phic[id], wgt) : q;
  // local part of RH at the cell (eigen-decomposition of Theta, Eqs. NS21-NS24)
  T dg[N], of[N == 2 ? 1 : 3], R[N][N], rl[NC];
  lcr_rhs_local<T, N>(th0, L, qc, rl, R, dg);
  const T dt = q.dt;
  T newth[NC];
#pragma unroll
  for (int cq = 0; cq < NC; ++cq) {
    const T rh = rl[cq] - adv[cq];
    const T t0 = th0[cq];
    newth[cq] = STAGE == 1 ? t0 + dt * rh : (T)0.5 * P.base[cq][id] + (T)0.5 * (t0 + dt * rh);
  }
#pragma unroll
  for (int cq = 0; cq < NC; ++cq) P.out[cq][id] = newth[cq];
  if (STAGE == 2) {
    // tau = (1 + phi)/2 (mu_p/lambda_H) (W e^theta W^T - I), W the eigenvectors of
    // Theta^{n+1}: in closed form in FP32 and FP64.  With Jacobi (the
    // derivative-carrying type), Theta^{n+1}, which differs from the stage's Theta
    // by O(dt), is first rotated into that Theta's eigenbasis R (R^T Theta^{n+1} R
    // is nearly diagonal and Jacobi converges in about a sweep); W = R V.
    if constexpr (N == 3 && !IsDual<T>::value) {
      dg[0] = newth[0], dg[1] = newth[1], dg[2] = newth[2];
      of[0] = newth[3], of[1] = newth[4], of[2] = newth[5];
      eig_sym<T, N>(dg, of, R);
    } else if constexpr (N == 3) {
      T A[N][N], B[N][N];
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) A[a][b] = newth[comp_of<N>(a, b)];
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
          T sab = 0;
#pragma unroll
          for (int c = 0; c < N; ++c) sab += A[a][c] * R[c][b];
          B[a][b] = sab;  // Theta^{n+1} R
        }
      auto rot = [&](int a, int b) {  // (R^T Theta^{n+1} R)_ab
        T sab = 0;
#pragma unroll
        for (int c = 0; c < N; ++c) sab += R[c][a] * B[c][b];
        return sab;
      };
      dg[0] = rot(0, 0);
      dg[1] = rot(1, 1);
      dg[2] = rot(2, 2);
      of[0] = rot(0, 1);
      of[1] = rot(0, 2);
      of[2] = rot(1, 2);
      T V[N][N];
      eig_sym<T, N>(dg, of, V);
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
          T sab = 0;
#pragma unroll
          for (int c = 0; c < N; ++c) sab += R[a][c] * V[c][b];
          B[a][b] = sab;
        }
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) R[a][b] = B[a][b];
    } else {
#pragma unroll
      for (int a = 0; a < N; ++a) dg[a] = newth[comp_of<N>(a, a)];
      of[0] = newth[comp_of<N>(0, 1)];
      eig_sym<T, N>(dg, of, R);
    }
    T ex[N];
#pragma unroll
    for (int c = 0; c < N; ++c) ex[c] = fexp<T>(dg[c]);
    if (!q.ap1) wgt = (T)0.5 * ((T)1 + P.phic[id]) * q.wtau;
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int b = a; b < N; ++b) {
        T s = 0;
#pragma unroll
        for (int c = 0; c < N; ++c) s += R[a][c] * ex[c] * R[b][c];
        P.tau[comp_of<N>(a, b)][id] = wgt * (s - (a == b ? (T)1 : (T)0));
      }
  }
}

template <class T, int N>
__device__ __forceinline__ void k_polymer_b(const PolyIn<T>& P, const Dims& d, const PhysT<T>& q, int stage, const int3 bid, unsigned char*) {
  RowIdx x;
  if (!row_index_b(bid, d.nx, d.ny, x)) return;
  if (stage == 1) polymer_cell<T, N, 1>(P, d, q, x);
  else polymer_cell<T, N, 2>(P, d, q, x);
}

// FP32: 64 registers, eight 128-thread CTAs per SM (with the closed-form
// eigen-decomposition, stage 1 measured 8 % and stage 2 2 % faster than at 48
// registers, and 5 % and 10 % faster than at 80).  The budget is fixed, not a
// tuning knob: the compiler's schedule, and so the rounding, differs between
// budgets.
template <class T, int N, int STAGE>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 8 : 1) k_polymer(const __grid_constant__ PolyIn<T> P, const Dims d, const PhysT<T> q) {
  RowIdx x;
  if (!row_index(d.nx, d.ny, x)) return;
  polymer_cell<T, N, STAGE>(P, d, q, x);
}

}  // namespace pf
