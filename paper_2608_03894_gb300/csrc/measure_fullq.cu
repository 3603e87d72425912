// Full-momentum maps of the two order-parameter correlators (Sec. III and
// IV) from one FP64 G, at every momentum Q = m1 b1 / L + m2 b2 / L of the mesh.
//
//   S_Pair(Q)     = (1/N) Re sum_ij e^{iQ(r_i - r_j)} X_ij,
//                   X_ij = (delta_ij - G_ij)^2 + G_ij^2
//   <phi+ phi>(Q) = (1/N^2) [ |sum_x w_x n_x|^2 + 2 Re sum_xy conj(w_x) w_y Y_xy ],
//                   n_x = 2 (1 - G_xx), Y_xy = (delta_xy - G_yx) G_xy,
//                   w_x = e^{iQ R_x} w^{a_x}, w = e^{2 pi i / 3}
// (the real part of the pair sum is the same with G_ij or G_ji in X, since
// swapping i and j conjugates the sum).
//
// Both sums depend on i, j only through the sublattices a, b and the cell
// difference D = R_i - R_j, so one pass over G bins them:
//   C_ab(D) = sum_R X_{(R,a),(R-D,b)},   Y_ab(D) = sum_R Y_{(R,a),(R-D,b)}
// (9 L^2 bins each; thread per bin, summing over R in a fixed order: the
// result does not depend on scheduling), and a second kernel takes the
// L x L Fourier sums per Q with phases from a table of e^{2 pi i k / (2L)}
// (all phases are multiples of 2 pi / (2L): the sublattice offsets are half
// cells):
//   S(Q)   = (1/N) Re sum_ab e^{iQ(tau_a - tau_b)} sum_D e^{iQ D} C_ab(D)
//   phi(Q) = (1/N^2) [ |sum_a w^a sum_R e^{iQR} n_(R,a)|^2
//                      + 2 Re sum_ab w^{b-a} sum_D e^{-iQ D} Y_ab(D) ].
// The binning pass reads G twice (G_ij and G_ji): it is bound by HBM.
#include <cmath>
#include <vector>

#include "kernels.cuh"

namespace dq {

__global__ void __launch_bounds__(256)
    fullq_bin_kernel(const double *__restrict__ G, int L, double *__restrict__ C, double *__restrict__ Y) {
  const int L2 = L * L, N = 3 * L2;
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;  // ((a * 3 + b) * L + d1) * L + d2
  if (bin >= 9 * L2) return;
  const int d2 = bin % L, d1 = (bin / L) % L, ab = bin / L2, a = ab / 3, b = ab % 3;
  double cx = 0.0, cy = 0.0;
  for (int r1 = 0; r1 < L; ++r1) {
    const int s1 = (r1 - d1 + L) % L;
    for (int r2 = 0; r2 < L; ++r2) {
      const int s2 = (r2 - d2 + L) % L;
      const int i = (r1 * L + r2) * 3 + a, j = (s1 * L + s2) * 3 + b;
      const double gij = G[(size_t)i * N + j], gji = G[(size_t)j * N + i];
      const double dl = (i == j) ? 1.0 : 0.0;
      cx += (dl - gij) * (dl - gij) + gij * gij;
      cy += (dl - gji) * gij;
    }
  }
  C[bin] = cx;
  Y[bin] = cy;
}

// one thread per momentum (m1, m2); ph[k] = e^{2 pi i k / (2L)}, k < 2L;
// off[a] = (f1, f2) offsets in half cells (site positions) or zeros
__global__ void __launch_bounds__(128)
    fullq_dft_kernel(const double *__restrict__ G, int L, const double *__restrict__ C,
                     const double *__restrict__ Yb, const double2 *__restrict__ ph, int offsets,
                     double *__restrict__ S, double *__restrict__ P) {
  const int L2 = L * L, N = 3 * L2, L2x = 2 * L;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= L2) return;
  const int m1 = q / L, m2 = q % L;
  // sublattice offsets tau_a in half cells: A (0, 0), B (0, -1), C (-1, 0)
  const int h1[3] = {0, 0, -1}, h2[3] = {0, -1, 0};
  double s_re = 0.0, y_re = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const int ab = a * 3 + b;
      double cr = 0.0, ci = 0.0, yr = 0.0, yi = 0.0;
      for (int d1 = 0; d1 < L; ++d1)
        for (int d2 = 0; d2 < L; ++d2) {
          const int k = (2 * ((m1 * d1 + m2 * d2) % L)) % L2x;  // e^{iQD}
          const double2 e = ph[k];
          const double c = C[(ab * L + d1) * L + d2], y = Yb[(ab * L + d1) * L + d2];
          cr = fma(e.x, c, cr);
          ci = fma(e.y, c, ci);
          yr = fma(e.x, y, yr);  // e^{-iQD} y: real part e.x y, imaginary -e.y y
          yi = fma(-e.y, y, yi);
        }
      // e^{iQ(tau_a - tau_b)} (site positions) and w^{b - a} = e^{2 pi i (b - a) / 3}
      int kt = 0;
      if (offsets) kt = ((m1 * (h1[a] - h1[b]) + m2 * (h2[a] - h2[b])) % L2x + L2x) % L2x;
      const double2 t = ph[kt];
      s_re += t.x * cr - t.y * ci;
      const double ang = 6.283185307179586476925286766559 * (double)(b - a) / 3.0;
      double sw, cw;
      sincos(ang, &sw, &cw);
      y_re += cw * yr - sw * yi;
    }
  // diagonal term: sum_a w^a sum_R e^{iQR} n_(R,a)
  double dr = 0.0, di = 0.0;
  for (int a = 0; a < 3; ++a) {
    double ar = 0.0, ai = 0.0;
    for (int r1 = 0; r1 < L; ++r1)
      for (int r2 = 0; r2 < L; ++r2) {
        const int x = (r1 * L + r2) * 3 + a;
        const double n = 2.0 * (1.0 - G[(size_t)x * N + x]);
        const double2 e = ph[(2 * ((m1 * r1 + m2 * r2) % L)) % L2x];
        ar = fma(e.x, n, ar);
        ai = fma(e.y, n, ai);
      }
    const double ang = 6.283185307179586476925286766559 * (double)a / 3.0;
    double sw, cw;
    sincos(ang, &sw, &cw);
    dr += cw * ar - sw * ai;
    di += sw * ar + cw * ai;
  }
  S[q] = s_re / N;
  P[q] = (dr * dr + di * di + 2.0 * y_re) / ((double)N * N);
}

}  // namespace dq

using namespace dq;

extern "C" dqmc_status dqmc_op_measure_fullq(int L, const double *G, int site_offsets, double *S_out,
                                             double *phi2_out, void *stream) try {
  if (!supported_L(L)) return fail(DQMC_EINVAL, "unsupported L");
  if (!G || !S_out || !phi2_out) return fail(DQMC_EINVAL, "null pointer");
  const int L2 = L * L;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<double> tab(4 * (size_t)L);
  for (int k = 0; k < 2 * L; ++k) {
    const double ang = 3.141592653589793238462643383279 * (double)k / L;
    tab[2 * k] = std::cos(ang);
    tab[2 * k + 1] = std::sin(ang);
  }
  // scratch: bins C, Y (9 L^2 each), the phase table (2L complex), outputs S, P (L^2 each)
  const size_t nd = 18 * (size_t)L2 + 4 * (size_t)L + 2 * (size_t)L2;
  double *d = nullptr;
  DQ_CUDA(cudaMallocAsync((void **)&d, nd * sizeof(double), st));
  double *C = d, *Yb = C + 9 * (size_t)L2, *ph = Yb + 9 * (size_t)L2, *S = ph + 4 * (size_t)L, *P = S + L2;
  cudaError_t e = cudaMemcpyAsync(ph, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    DQ_KSCOPE(KF_MEASURE, st);
    add_work(KF_MEASURE, 8.0 * 3.0 * L2 * 3.0 * L2, 2.0 * 8.0 * 9.0 * L2 * (double)L2);
    fullq_bin_kernel<<<(9 * L2 + 255) / 256, 256, 0, st>>>(G, L, C, Yb);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    DQ_KSCOPE(KF_MEASURE, st);
    fullq_dft_kernel<<<(L2 + 127) / 128, 128, 0, st>>>(G, L, C, Yb, reinterpret_cast<const double2 *>(ph),
                                                      site_offsets ? 1 : 0, S, P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(S_out, S, (size_t)L2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(phi2_out, P, (size_t)L2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  const cudaError_t e2 = cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "dqmc_op_measure_fullq");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
  return DQMC_OK;
} DQ_API_CATCH
