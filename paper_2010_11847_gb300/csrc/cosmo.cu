// cosmo.cu -- FP64 time-stepping coefficients and sigma8 normalisation.
//
// The only FP64 arithmetic of the library lives here: the linear growth
// D1, second-order growth D2, their logarithmic rates, the FastPM kick and
// drift factors of the leapfrog (Eqs. 1-2 with the growth-factor form of
// FastPM), and the sigma8 normalisation of the Eisenstein & Hu (1998)
// no-wiggle spectrum.  Everything runs on the GPU so that a whole run,
// including its coefficients, is stream-ordered.
#include "internal.h"

#include <math.h>

namespace fpm {

constexpr double A_INIT = 1e-5;    // growing-mode start: D1 = a, D2 = -3/7 a^2

struct GrowthCoef {
  double c1, c2;   // D'' = -c1 D' + c2 (D - D1^2 for D2), c1 = 2 + dlnE/dlna, c2 = 1.5 Om(a)
};

__device__ __forceinline__ GrowthCoef growth_coef(double a, double om) {
  const double ainv3 = 1.0 / (a * a * a);
  const double om_a = om * ainv3 / (om * ainv3 + (1.0 - om));
  GrowthCoef c;
  c.c1 = 2.0 - 1.5 * om_a;
  c.c2 = 1.5 * om_a;
  return c;
}

__device__ __forceinline__ void growth_rhs(const GrowthCoef& c, const double* y, double* dy) {
  dy[0] = y[1];
  dy[1] = -c.c1 * y[1] + c.c2 * y[0];
  dy[2] = y[3];
  dy[3] = -c.c1 * y[3] + c.c2 * (y[2] - y[0] * y[0]);
}

// One CTA per scale factor a_in[0..n]; a_in[n] must be 1 (the
// normalisation point).  raw[4*i..]: D1, dD1/dlna, D2, dD2/dlna unnormalised.
// Each target integrates from A_INIT with RK4_CHAIN RK4 steps of size h in
// ln a.  The ODE coefficients at the 2*RK4_CHAIN+1 half-step points do not
// depend on the solution and are computed by the whole CTA first.  The
// chain is then evaluated in parallel, with the same discretisation: the
// D1 system is linear, so each RK4 step is a 2x2 matrix A_s (the same
// matrix acts on the homogeneous part of D2); an exclusive prefix scan of
// the A_s gives D1 at every step start, from which each step's D2 source
// increment b_s follows; the D2 steps are affine maps y -> A_s y + b_s,
// composed by an ordered reduction.  Only the association of the FP64
// products differs from the serial chain.
constexpr int RK4_CHAIN = 1024;
constexpr int GROWTH_THREADS = 256;
constexpr int STEPS_PER_THREAD = RK4_CHAIN / GROWTH_THREADS;

struct M2 {
  double a, b, c, d;   // [[a b] [c d]]
};
__device__ __forceinline__ M2 mmul(const M2& x, const M2& y) {   // x * y
  return M2{x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
__device__ __forceinline__ void mvec(const M2& m, double u, double v, double* ou, double* ov) {
  *ou = m.a * u + m.b * v;
  *ov = m.c * u + m.d * v;
}

// One RK4 step of the 4-state system from y (D1, D1', D2, D2'); the D2
// source uses the D1 stage values, as the serial chain does.
__device__ __forceinline__ void rk4_step(const GrowthCoef& cs, const GrowthCoef& cm, const GrowthCoef& ce, double h,
                                         double* y) {
  double k1[4], k2[4], k3[4], k4[4], t[4];
  growth_rhs(cs, y, k1);
  for (int i = 0; i < 4; ++i) t[i] = y[i] + 0.5 * h * k1[i];
  growth_rhs(cm, t, k2);
  for (int i = 0; i < 4; ++i) t[i] = y[i] + 0.5 * h * k2[i];
  growth_rhs(cm, t, k3);
  for (int i = 0; i < 4; ++i) t[i] = y[i] + h * k3[i];
  growth_rhs(ce, t, k4);
  for (int i = 0; i < 4; ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

__global__ void __launch_bounds__(GROWTH_THREADS) k_growth_raw(const double* __restrict__ a_in, double om,
                                                               double* __restrict__ raw) {
  __shared__ double c1[2 * RK4_CHAIN + 1], c2[2 * RK4_CHAIN + 1];
  __shared__ double scratch[GROWTH_THREADS * 6];
  M2* pre = reinterpret_cast<M2*>(scratch);                         // D1 scan: products of each thread's steps
  double(*aff)[6] = reinterpret_cast<double(*)[6]>(scratch);      // then the D2 reduction: affine maps (M2, b)
  const double lna0 = log(A_INIT);
  const double h = (log(a_in[blockIdx.x]) - lna0) / RK4_CHAIN;
  for (int j = threadIdx.x; j <= 2 * RK4_CHAIN; j += blockDim.x) {
    const GrowthCoef c = growth_coef(exp(lna0 + 0.5 * h * j), om);
    c1[j] = c.c1;
    c2[j] = c.c2;
  }
  __syncthreads();
  const int tid = threadIdx.x, s0 = tid * STEPS_PER_THREAD;
  auto coefs = [&](int s, GrowthCoef* cs, GrowthCoef* cm, GrowthCoef* ce) {
    *cs = GrowthCoef{c1[2 * s], c2[2 * s]};
    *cm = GrowthCoef{c1[2 * s + 1], c2[2 * s + 1]};
    *ce = GrowthCoef{c1[2 * s + 2], c2[2 * s + 2]};
  };
  // step matrices of the linear part: the RK4 step applied to the unit vectors
  M2 A[STEPS_PER_THREAD];
#pragma unroll
  for (int q = 0; q < STEPS_PER_THREAD; ++q) {
    GrowthCoef cs, cm, ce;
    coefs(s0 + q, &cs, &cm, &ce);
    double e1[4] = {1.0, 0.0, 0.0, 0.0}, e2[4] = {0.0, 1.0, 0.0, 0.0};
    rk4_step(cs, cm, ce, h, e1);
    rk4_step(cs, cm, ce, h, e2);
    A[q] = M2{e1[0], e2[0], e1[1], e2[1]};
  }
  // exclusive scan of the products (later steps multiply from the left)
  M2 local = A[0];
#pragma unroll
  for (int q = 1; q < STEPS_PER_THREAD; ++q) local = mmul(A[q], local);
  pre[tid] = local;
  __syncthreads();
  for (int off = 1; off < GROWTH_THREADS; off <<= 1) {   // inclusive Hillis-Steele: pre[t] = P(t) ... P(0)
    const M2 other = tid >= off ? pre[tid - off] : M2{1.0, 0.0, 0.0, 1.0};
    __syncthreads();
    pre[tid] = mmul(pre[tid], other);
    __syncthreads();
  }
  const M2 before = tid ? pre[tid - 1] : M2{1.0, 0.0, 0.0, 1.0};
  __syncthreads();                              // pre is reused as aff below
  // D1 state at each of this thread's step starts; D2 source increments
  const double a0 = A_INIT;
  double u, v;
  mvec(before, a0, a0, &u, &v);                 // y1 = (D1, D1') at step s0
  M2 Q{1.0, 0.0, 0.0, 1.0};
  double bu = 0.0, bv = 0.0;                    // this thread's composed D2 affine map: y2 -> Q y2 + (bu, bv)
#pragma unroll
  for (int q = 0; q < STEPS_PER_THREAD; ++q) {
    GrowthCoef cs, cm, ce;
    coefs(s0 + q, &cs, &cm, &ce);
    double y[4] = {u, v, 0.0, 0.0};
    rk4_step(cs, cm, ce, h, y);                 // D2 part: the source increment b_s (zero D2 start)
    double nu, nv;
    mvec(A[q], bu, bv, &nu, &nv);
    bu = nu + y[2];
    bv = nv + y[3];
    Q = mmul(A[q], Q);
    u = y[0];
    v = y[1];
  }
  aff[tid][0] = Q.a; aff[tid][1] = Q.b; aff[tid][2] = Q.c; aff[tid][3] = Q.d;
  aff[tid][4] = bu; aff[tid][5] = bv;
  __syncthreads();
  // ordered reduction: (Q2, b2) after (Q1, b1) = (Q2 Q1, Q2 b1 + b2)
  for (int w = 1; w < GROWTH_THREADS; w <<= 1) {
    if ((tid & (2 * w - 1)) == 0) {
      const double* L = aff[tid];
      const double* R = aff[tid + w];
      const M2 q1{L[0], L[1], L[2], L[3]}, q2{R[0], R[1], R[2], R[3]};
      const M2 q = mmul(q2, q1);
      double nu, nv;
      mvec(q2, L[4], L[5], &nu, &nv);
      aff[tid][0] = q.a; aff[tid][1] = q.b; aff[tid][2] = q.c; aff[tid][3] = q.d;
      aff[tid][4] = nu + R[4];
      aff[tid][5] = nv + R[5];
    }
    __syncthreads();
  }
  if (tid == GROWTH_THREADS - 1) {              // the last thread holds D1 at the end of the chain
    const M2 q{aff[0][0], aff[0][1], aff[0][2], aff[0][3]};
    double d2u, d2v;
    mvec(q, -3.0 / 7.0 * a0 * a0, -6.0 / 7.0 * a0 * a0, &d2u, &d2v);
    raw[4 * blockIdx.x + 0] = u;
    raw[4 * blockIdx.x + 1] = v;
    raw[4 * blockIdx.x + 2] = d2u + aff[0][4];
    raw[4 * blockIdx.x + 3] = d2v + aff[0][5];
  }
}

// out[6*i..]: D1, D2, f1, f2, E, dD1/da, normalised by row n (a = 1).
__global__ void k_growth_norm(const double* __restrict__ a_in, const double* __restrict__ raw, int n,
                              double om, double* __restrict__ out) {
  const int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i >= n) return;
  const double norm = raw[4 * n];
  const double* y = raw + 4 * i;
  const double a = a_in[i];
  double* o = out + 6 * i;
  o[0] = y[0] / norm;
  o[1] = y[2] / (norm * norm);
  o[2] = y[1] / y[0];
  o[3] = y[3] / y[2];
  o[4] = sqrt(om / (a * a * a) + (1.0 - om));
  o[5] = y[1] / norm / a;
}

// FastPM factors from growth values at stages a_0..a_n (rows 0..n) and half
// stages a_h (rows n+1..2n), written to fac[3*k + {0,1,2}] = kick1, drift, kick2:
//   drift a_i->a_f, p at a_c: (D1(a_f)-D1(a_i)) / (a_c^3 E(a_c) dD1/da(a_c))
//   kick  a_i->a_f, f at a_c: (G_f(a_f)-G_f(a_i)) / (a_c^2 E(a_c) g_f(a_c)),
//   G_f = a^3 E dD1/da, g_f = 1.5 Om D1 / (a^2 E).
__global__ void k_factors(const double* __restrict__ a_pts, const double* __restrict__ gr, int nsteps,
                          double om, double* __restrict__ fac) {
  const int k = threadIdx.x + blockIdx.x * blockDim.x;
  if (k >= nsteps) return;
  auto D1 = [&](int r) { return gr[6 * r + 0]; };
  auto E = [&](int r) { return gr[6 * r + 4]; };
  auto dD = [&](int r) { return gr[6 * r + 5]; };
  auto A = [&](int r) { return a_pts[r]; };
  auto Gf = [&](int r) { return A(r) * A(r) * A(r) * E(r) * dD(r); };
  auto gf = [&](int r) { return 1.5 * om * D1(r) / (A(r) * A(r) * E(r)); };
  const int i0 = k, i1 = k + 1, ih = nsteps + 1 + k;
  fac[3 * k + 0] = (Gf(ih) - Gf(i0)) / (A(i0) * A(i0) * E(i0) * gf(i0));
  fac[3 * k + 1] = (D1(i1) - D1(i0)) / (A(ih) * A(ih) * A(ih) * E(ih) * dD(ih));
  fac[3 * k + 2] = (Gf(i1) - Gf(ih)) / (A(i1) * A(i1) * E(i1) * gf(i1));
}

// ------------------------------------------------------------ sigma8
__device__ double eh_nowiggle_T64(double k_h, const CosmoParams& c) {
  const double theta = c.t_cmb / 2.7;
  const double wm = c.omega_m * c.h * c.h, wb = c.omega_b * c.h * c.h;
  const double fb = c.omega_b / c.omega_m;
  const double s = 44.5 * log(9.83 / wm) / sqrt(1.0 + 10.0 * pow(wb, 0.75));
  const double alpha = 1.0 - 0.328 * log(431.0 * wm) * fb + 0.38 * log(22.3 * wm) * fb * fb;
  const double ks = 0.43 * k_h * c.h * s;
  const double ks2 = ks * ks;
  const double gamma = c.omega_m * c.h * (alpha + (1.0 - alpha) / (1.0 + ks2 * ks2));
  const double q = k_h * theta * theta / gamma;
  const double L0 = log(2.0 * 2.718281828459045235 + 1.8 * q);
  const double C0 = 14.2 + 731.0 / (1.0 + 62.5 * q);
  return L0 / (L0 + C0 * q * q);
}

// sigma(8 Mpc/h)^2 of P = k^ns T^2 (unit amplitude): Simpson's rule on a
// uniform ln k grid of SIGMA_PTS points over [1e-5, 1e2] h/Mpc.  One block;
// a fixed-order tree reduction keeps the sum deterministic.  Writes
// amp[0] = sigma8^2 / that integral.
constexpr int SIGMA_PTS = 4097;
constexpr int SIGMA_THREADS = 512;
__global__ void __launch_bounds__(SIGMA_THREADS) k_sigma8(CosmoParams c, double* __restrict__ amp) {
  __shared__ double part[SIGMA_THREADS];
  const double lk0 = log(1e-5), lk1 = log(1e2);
  const double dl = (lk1 - lk0) / (SIGMA_PTS - 1);
  double acc = 0.0;
  for (int i = threadIdx.x; i < SIGMA_PTS; i += SIGMA_THREADS) {
    const double k = exp(lk0 + dl * i);
    const double x = 8.0 * k;
    const double w = 3.0 * (sin(x) - x * cos(x)) / (x * x * x);
    const double T = eh_nowiggle_T64(k, c);
    const double f = k * k * k * pow(k, c.n_s) * T * T * w * w;
    const double sw = (i == 0 || i == SIGMA_PTS - 1) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    acc += sw * f;
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int s = SIGMA_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sig2 = dl / 3.0 * part[0] / (2.0 * 3.14159265358979323846 * 3.14159265358979323846);
    amp[0] = c.sigma8 * c.sigma8 / sig2;
  }
}

// ------------------------------------------------------------ host side
int launch_sigma8(const CosmoParams& c, double* d_amp, cudaStream_t s) {
  k_sigma8<<<1, SIGMA_THREADS, 0, s>>>(c, d_amp);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

// d_a holds n scale factors followed by a_n = 1 (n+1 values); d_raw has
// room for 4*(n+1) doubles; d_out receives 6*n doubles.
int launch_growth(const double* d_a, int n, double om, double* d_raw, double* d_out, cudaStream_t s) {
  if (n <= 0) return FPM_OK;
  const int threads = 64;
  k_growth_raw<<<n + 1, GROWTH_THREADS, 0, s>>>(d_a, om, d_raw);
  FPM_CUDA_TRY(cudaGetLastError());
  k_growth_norm<<<(n + threads - 1) / threads, threads, 0, s>>>(d_a, d_raw, n, om, d_out);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

// d_pts holds a_0..a_n, then the half stages, then 1.0 (2n+2 values,
// filled by the caller); d_raw / d_gr receive the raw and normalised growth
// rows, d_fac the factors.
int launch_factors(const double* d_pts, int nsteps, double om, double* d_raw, double* d_gr,
                   double* d_fac, cudaStream_t s) {
  FPM_TRY(launch_growth(d_pts, 2 * nsteps + 1, om, d_raw, d_gr, s));
  if (nsteps > 0) {
    k_factors<<<(nsteps + 127) / 128, 128, 0, s>>>(d_pts, d_gr, nsteps, om, d_fac);
    FPM_CUDA_TRY(cudaGetLastError());
  }
  return FPM_OK;
}

}  // namespace fpm
