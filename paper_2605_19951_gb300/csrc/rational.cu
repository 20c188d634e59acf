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
                                                           double *__restrict__ Y, double2 *__restrict__ alpha) {
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
  if (threadIdx.x == 0) {
    for (int i = ncol - 1; i >= 0; i--) {
      double s = y[i];
      for (int q = i + 1; q < ncol; q++) s -= B[int64_t(q) * rows + i] * coef[q];
      coef[i] = s / rdiag[i];
    }
    for (int i = 0; i < m; i++) alpha[int64_t(i) * K + j] = make_double2(coef[i], coef[m + i]);
  }
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
                      const double *cf, const double *t, int K, double *Y, double2 *alpha, cudaStream_t s) {
  tem::count_launch();
  k_fit_solve<<<K, kFitThreads, 0, s>>>(B, nz + 1 + 2 * m, m, nz, lz0, lz1, rdiag, cf, t, K, Y, alpha);
}

}  // namespace tem
