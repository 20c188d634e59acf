// Residues of the rational approximant for a set of observation times
// (Section 2.3): the poles xi_i are shared by every time t_j, and only the
// coefficients alpha_i^[j] of
//   r_j(z) = 2 Re sum_i alpha_i^[j] / (z - xi_i)   ~   exp(-t_j z)
// depend on t_j.  With the poles fixed they are a linear least-squares
// problem per time over a sample set of z on the non-negative real axis
// (where the spectrum of M^-1 K lies), with a Tikhonov term
// mu alpha_i / |xi_i| that bounds each partial fraction (max over z >= 0 of
// |alpha_i / (z - xi_i)| is |alpha_i| / |xi_i| for Re xi_i < 0).  Unknowns
// are (Re alpha_i, Im alpha_i); the basis columns are 2 Re c_i and
// -2 Im c_i with c_i = 1 / (z - xi_i).
//
// All in FP64 on the device: the (n_z + 1 + 2m) x 2m matrix (sample rows z = 0
// and n_z log-spaced points, then the 2m Tikhonov rows) is reduced once by
// Householder QR (one CTA), and every time's right-hand side exp(-t_j z)
// (zero on the Tikhonov rows) is reduced by the same reflections and solved
// against R by one CTA per time.
#include "common.cuh"
#include "kernels.h"

namespace tem {

namespace {
constexpr int kFitThreads = 512;

// z of sample row r: 0, then 10^(lz0 + (r - 1) dlz) for r = 1 .. nz (the last exactly 10^lz1)
__device__ __forceinline__ double sample_z(int64_t r, int64_t nz, double lz0, double lz1) {
  if (r == 0) return 0.0;
  if (r == nz) return pow(10.0, lz1);
  const double dl = nz > 1 ? (lz1 - lz0) / double(nz - 1) : 0.0;
  return pow(10.0, lz0 + double(r - 1) * dl);
}

// block sum over all threads of the CTA (kFitThreads)
__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();   // red is free again
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < kFitThreads / 32; q++) s += red[q];   // same order in every thread
  return s;
}
}  // namespace

// B column-major [rows][ncol], rows = nz + 1 + ncol, ncol = 2m.
__global__ void k_fit_basis(const double2 *__restrict__ xi, int m, int64_t nz, double lz0, double lz1, double mu,
                            double *__restrict__ B) {
  const int64_t rows = nz + 1 + 2 * m;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < rows * 2 * m;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e % rows;
    const int col = int(e / rows), i = col % m;
    double v = 0.0;
    if (r <= nz) {
      // c = 1 / (z - xi) = (z - xr + i xq) / |z - xi|^2 for xi = xr + i xq
      const double z = sample_z(r, nz, lz0, lz1);
      const double a = z - xi[i].x, b = -xi[i].y;   // z - xi = a + i b
      const double d = a * a + b * b;
      v = col < m ? 2.0 * a / d : 2.0 * b / d;      // 2 Re c, -2 Im c = 2 b / d
    } else if (r - nz - 1 == col) {
      v = mu / sqrt(xi[i].x * xi[i].x + xi[i].y * xi[i].y);
    }
    B[e] = v;
  }
}

// Householder QR of B in place (one CTA).  Column j's reflector is
// H_j = I - c_j v v^T, v = x - a e_j over rows j.., x = B[j.., j],
// a = -sign(x_j) |x|, c_j = 1 / (|x| (|x| + |x_j|)); v is stored in
// B[j.., j], a (the diagonal of R) in rdiag[j], c_j in cf[j]; the strict
// upper triangle of R overwrites B above the diagonal.
__global__ void __launch_bounds__(kFitThreads) k_fit_qr(double *__restrict__ B, int64_t rows, int ncol,
                                                        double *__restrict__ rdiag, double *__restrict__ cf) {
  __shared__ double red[kFitThreads / 32];
  __shared__ double sh_c;
  for (int j = 0; j < ncol; j++) {
    double *x = B + int64_t(j) * rows;
    double s2 = 0.0;
    for (int64_t r = j + 1 + threadIdx.x; r < rows; r += kFitThreads) s2 += x[r] * x[r];
    s2 = block_sum(s2, red);
    if (threadIdx.x == 0) {
      const double x0 = x[j], nx = sqrt(x0 * x0 + s2);
      double c = 0.0, a = 0.0;
      if (nx > 0.0) {
        a = x0 >= 0.0 ? -nx : nx;
        c = 1.0 / (nx * (nx + fabs(x0)));
        x[j] = x0 - a;
      }
      rdiag[j] = a;
      cf[j] = c;
      sh_c = c;
    }
    __syncthreads();
    const double c = sh_c;
    for (int q = j + 1; q < ncol; q++) {
      double *y = B + int64_t(q) * rows;
      double d = 0.0;
      for (int64_t r = j + threadIdx.x; r < rows; r += kFitThreads) d += x[r] * y[r];
      d = c * block_sum(d, red);
      for (int64_t r = j + threadIdx.x; r < rows; r += kFitThreads) y[r] -= d * x[r];
      __syncthreads();
    }
  }
}

// One CTA per time t_j: y = exp(-t_j z) on the sample rows, 0 on the
// Tikhonov rows (work column Y[j]); y = H_{ncol-1} .. H_0 y; R coef = y[0..ncol);
// alpha[i][j] = (coef[i], coef[m + i]).
__global__ void __launch_bounds__(kFitThreads) k_fit_solve(const double *__restrict__ B, int64_t rows, int m,
                                                           int64_t nz, double lz0, double lz1,
                                                           const double *__restrict__ rdiag,
                                                           const double *__restrict__ cf,
                                                           const double *__restrict__ t, int K,
                                                           double *__restrict__ Y, double2 *__restrict__ alpha,
                                                           double *__restrict__ coef_out,
                                                           double *__restrict__ tail_sq) {
  __shared__ double red[kFitThreads / 32];
  __shared__ double coef[64];
  const int j = blockIdx.x, ncol = 2 * m;
  double *y = Y + int64_t(j) * rows;
  const double tj = t[j];
  for (int64_t r = threadIdx.x; r < rows; r += kFitThreads)
    y[r] = r <= nz ? exp(-tj * sample_z(r, nz, lz0, lz1)) : 0.0;
  __syncthreads();
  for (int q = 0; q < ncol; q++) {
    const double *v = B + int64_t(q) * rows;
    double d = 0.0;
    for (int64_t r = q + threadIdx.x; r < rows; r += kFitThreads) d += v[r] * y[r];
    d = cf[q] * block_sum(d, red);
    for (int64_t r = q + threadIdx.x; r < rows; r += kFitThreads) y[r] -= d * v[r];
    __syncthreads();
  }
  if (tail_sq) {   // the least-squares residual: the part of Q^T e beyond the first ncol rows
    double ss = 0.0;
    for (int64_t r = ncol + threadIdx.x; r < rows; r += kFitThreads) ss += y[r] * y[r];
    ss = block_sum(ss, red);
    if (threadIdx.x == 0) tail_sq[j] = ss;
  }
  if (threadIdx.x == 0) {
    for (int i = ncol - 1; i >= 0; i--) {
      double s = y[i];
      for (int q = i + 1; q < ncol; q++) s -= B[int64_t(q) * rows + i] * coef[q];
      coef[i] = s / rdiag[i];
    }
    if (alpha)
      for (int i = 0; i < m; i++) alpha[int64_t(i) * K + j] = make_double2(coef[i], coef[m + i]);
    if (coef_out)
      for (int i = 0; i < ncol; i++) coef_out[int64_t(i) * K + j] = coef[i];
  }
}

// Variable projection (the poles as the unknowns, the residues eliminated by
// least squares): Kaufman's Jacobian of the residual r_j = (I - Q Q^T) e_j
// with respect to parameter q is -(I - Q Q^T) (dB/dp_q) c_j, c_j the
// coefficients of time j.  With p_i = log(-Re xi_i) and p_{m+i} = log(Im xi_i),
// dxi_i/dp_i = Re xi_i and dxi_i/dp_{m+i} = i Im xi_i; only the two columns of
// pole i depend on them: d(2 Re c)/dp = 2 Re(c^2 dxi), d(-2 Im c)/dp =
// -2 Im(c^2 dxi) with c = 1/(z - xi), and the penalty rows mu / |xi_i| give
// -mu Re(conj(xi_i) dxi) / |xi_i|^3.  One CTA per (parameter q, time j): the
// vector (dB/dp_q) c_j, reduced by Q^T, keeps its rows beyond ncol (the
// projection's range, in the rotated basis) in T[(j * 2m + q) * rows ...].
__global__ void __launch_bounds__(kFitThreads) k_vp_jac(const double *__restrict__ B, int64_t rows, int m,
                                                        int64_t nz, double lz0, double lz1, double mu,
                                                        const double2 *__restrict__ xi,
                                                        const double *__restrict__ cf,
                                                        const double *__restrict__ coef, int K,
                                                        double *__restrict__ T) {
  __shared__ double red[kFitThreads / 32];
  const int ncol = 2 * m, q = blockIdx.x, j = blockIdx.y, i = q % m;
  double *g = T + (int64_t(j) * ncol + q) * rows;
  const double xr = xi[i].x, xq = xi[i].y;
  // dxi/dp = (dr, di)
  const double dr = q < m ? xr : 0.0, di = q < m ? 0.0 : xq;
  const double ca = coef[int64_t(i) * K + j], cb = coef[int64_t(m + i) * K + j];
  for (int64_t r = threadIdx.x; r < rows; r += kFitThreads) {
    double v = 0.0;
    if (r <= nz) {
      const double z = sample_z(r, nz, lz0, lz1);
      const double a = z - xr, b = -xq, d = a * a + b * b;   // z - xi = a + i b, c = (a - i b) / d
      const double cr = a / d, ci = -b / d;
      const double sr = cr * cr - ci * ci, si = 2.0 * cr * ci;   // c^2
      const double wr = sr * dr - si * di, wi = sr * di + si * dr;   // c^2 dxi
      v = 2.0 * wr * ca - 2.0 * wi * cb;
    } else if (r - nz - 1 == i || r - nz - 1 == m + i) {
      const double n2 = xr * xr + xq * xq;
      const double dpen = -mu * (xr * dr + xq * di) / (n2 * sqrt(n2));
      v = dpen * (r - nz - 1 == i ? ca : cb);
    }
    g[r] = v;
  }
  __syncthreads();
  for (int h = 0; h < ncol; h++) {
    const double *v = B + int64_t(h) * rows;
    double d = 0.0;
    for (int64_t r = h + threadIdx.x; r < rows; r += kFitThreads) d += v[r] * g[r];
    d = cf[h] * block_sum(d, red);
    for (int64_t r = h + threadIdx.x; r < rows; r += kFitThreads) g[r] -= d * v[r];
    __syncthreads();
  }
}

// Normal equations of the Levenberg-Marquardt step from the projected tails:
// G[a][b] = sum_j <T_aj, T_bj> (a, b < ncol) and G[a][ncol] = sum_j <T_aj, Y_j>
// over the rows beyond ncol; one CTA per (a, b) with b <= ncol.
__global__ void __launch_bounds__(kFitThreads) k_vp_gram(const double *__restrict__ T,
                                                         const double *__restrict__ Y, int64_t rows, int ncol,
                                                         int K, double *__restrict__ G) {
  __shared__ double red[kFitThreads / 32];
  const int a = blockIdx.x, b = blockIdx.y;
  if (b < a && b < ncol) return;
  double s = 0.0;
  for (int j = 0; j < K; j++) {
    const double *ta = T + (int64_t(j) * ncol + a) * rows;
    const double *tb = b < ncol ? T + (int64_t(j) * ncol + b) * rows : Y + int64_t(j) * rows;
    for (int64_t r = ncol + threadIdx.x; r < rows; r += kFitThreads) s += ta[r] * tb[r];
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) G[a * (ncol + 1) + b] = s;
}

void launch_fit_qr(const double2 *xi, int m, int64_t nz, double lz0, double lz1, double mu, double *B,
                   double *rdiag, double *cf, cudaStream_t s) {
  const int64_t rows = nz + 1 + 2 * m;
  tem::count_launch();
  k_fit_basis<<<(unsigned)std::min<int64_t>(div_up(rows * 2 * m, 256), 4096), 256, 0, s>>>(xi, m, nz, lz0, lz1, mu,
                                                                                          B);
  tem::count_launch();
  k_fit_qr<<<1, kFitThreads, 0, s>>>(B, rows, 2 * m, rdiag, cf);
}

void launch_fit_solve(const double *B, int m, int64_t nz, double lz0, double lz1, const double *rdiag,
                      const double *cf, const double *t, int K, double *Y, double2 *alpha, cudaStream_t s,
                      double *coef, double *tail_sq) {
  tem::count_launch();
  k_fit_solve<<<K, kFitThreads, 0, s>>>(B, nz + 1 + 2 * m, m, nz, lz0, lz1, rdiag, cf, t, K, Y, alpha, coef,
                                        tail_sq);
}

void launch_vp_normal(const double *B, int m, int64_t nz, double lz0, double lz1, double mu, const double2 *xi,
                      const double *cf, const double *coef, int K, const double *Y, double *T, double *G,
                      cudaStream_t s) {
  const int64_t rows = nz + 1 + 2 * m;
  tem::count_launch();
  k_vp_jac<<<dim3(2 * m, K), kFitThreads, 0, s>>>(B, rows, m, nz, lz0, lz1, mu, xi, cf, coef, K, T);
  tem::count_launch();
  k_vp_gram<<<dim3(2 * m, 2 * m + 1), kFitThreads, 0, s>>>(T, Y, rows, 2 * m, K, G);
}

}  // namespace tem
