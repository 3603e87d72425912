// Equal-time estimators from one FP64 G in a single tiled pass.
//
// With X_rc = (delta_rc - G_rc)^2 + G_rc^2 (symmetric pair definition of
// Sec. III) and phase tables of the momenta:
//   S(Q)        = (1/N) sum_rc Re(p_c conj(p_r)) X_rc
//   <phi+phi>(Q)= (1/N^2) [ 4 |sum_x w_x (1 - G_xx)|^2
//                          + 2 sum_xy Re(conj(w_x) w_y) (delta_xy - G_yx) G_xy ]   (Sec. IV)
//   rho         = (2/N) sum_x (1 - G_xx)
//   E_kin       = (2/N) sum_ij K_ij (delta_ij - G_ji)
// Each CTA takes a 32 x 32 tile of G and the transposed tile (for G_yx).
#include "kernels.cuh"

namespace dq {


// raw[0..] : S_G, S_dk, cdwG_2nd, cdwK_2nd, diagG_re, diagG_im, diagK_re, diagK_im, dens, kin

__global__ void measure_tile_kernel(const double *__restrict__ G, int N, MeasTables t, double *raw) {
  __shared__ double tile[32][33];
  __shared__ double tileT[32][33];
  __shared__ double red[4][8];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;  // tile rows by.., cols bx..
  const int tx = threadIdx.x, ty = threadIdx.y;           // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int i = by + r, j = bx + tx;
    tile[r][tx] = (i < N && j < N) ? G[(size_t)i * N + j] : 0.0;
    const int i2 = bx + r, j2 = by + tx;  // transposed tile: G[bx + r][by + tx]
    tileT[r][tx] = (i2 < N && j2 < N) ? G[(size_t)i2 * N + j2] : 0.0;
  }
  __syncthreads();
  double sG = 0.0, sdk = 0.0, cg = 0.0, ck = 0.0;
  const int c = bx + tx;
  for (int r = ty; r < 32; r += 8) {
    const int rr = by + r;
    if (rr >= N || c >= N) continue;
    const double g = tile[r][tx];
    const double gt = tileT[tx][r];  // G[c][rr]
    const double d = (rr == c) ? 1.0 : 0.0;
    const double X = (d - g) * (d - g) + g * g;
    sG += X;
    sdk += (t.pc[rr] * t.pc[c] + t.ps[rr] * t.ps[c]) * X;
    const double dg = (d - gt) * g;
    cg += (t.wgc[rr] * t.wgc[c] + t.wgs[rr] * t.wgs[c]) * dg;
    if (t.wkc) ck += (t.wkc[rr] * t.wkc[c] + t.wks[rr] * t.wks[c]) * dg;
  }
  double v[4] = {sG, sdk, cg, ck};
#pragma unroll
  for (int q = 0; q < 4; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  if (tx == 0)
    for (int q = 0; q < 4; ++q) red[q][ty] = v[q];
  __syncthreads();
  if (ty == 0 && tx < 4) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[tx][w];
    atomicAdd(raw + tx, s);
  }
}

__global__ void measure_diag_kernel(const double *__restrict__ G, int N, MeasTables t, double *raw) {
  double a[6] = {0, 0, 0, 0, 0, 0};
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
    const double dx = 1.0 - G[(size_t)x * N + x];
    a[0] += t.wgc[x] * dx;
    a[1] += t.wgs[x] * dx;
    if (t.wkc) {
      a[2] += t.wkc[x] * dx;
      a[3] += t.wks[x] * dx;
    }
    a[4] += dx;
    double kin = 0.0;  // sum_j K_xj (delta - G_jx) = t * sum_nbr G_jx  (K = -t, off-diagonal)
    for (int q = 0; q < 4; ++q) kin += G[(size_t)t.nbr[4 * x + q] * N + x];
    a[5] += kin;
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    for (int o = 16; o > 0; o >>= 1) a[q] += __shfl_down_sync(0xffffffffu, a[q], o);
    if ((threadIdx.x & 31) == 0) atomicAdd(raw + 4 + q, a[q]);
  }
}

// obs[6] from raw sums (hopping t folded into the kinetic sum by the caller's table: K_ij = -t)
__global__ void measure_finalize_kernel(const double *raw, int N, double thop, int haveK, double *obs) {
  const double n = (double)N;
  obs[0] = raw[0] / n;
  obs[1] = raw[1] / n;
  obs[2] = (4.0 * (raw[4] * raw[4] + raw[5] * raw[5]) + 2.0 * raw[2]) / (n * n);
  obs[3] = haveK ? (4.0 * (raw[6] * raw[6] + raw[7] * raw[7]) + 2.0 * raw[3]) / (n * n)
                 : __longlong_as_double(0x7ff8000000000000ll);
  obs[4] = 2.0 * raw[8] / n;
  // sum_ij K_ij (delta_ij - G_ji) = -t sum_{x, nbr j} (-G_jx) = t sum G_jx
  obs[5] = 2.0 * thop * raw[9] / n;
}

cudaError_t launch_measure(const double *G, int N, const MeasTables &t, double *raw, double thop,
                           double *obs, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(raw, 0, kMeasRaw * sizeof(double), st);
  if (e != cudaSuccess) return e;
  dim3 grid((N + 31) / 32, (N + 31) / 32), block(32, 8);
  DQ_KSCOPE(KF_MEASURE, st);
  add_work(KF_MEASURE, 12.0 * N * (double)N, 8.0 * N * (double)N);
  measure_tile_kernel<<<grid, block, 0, st>>>(G, N, t, raw);
  DQ_KSCOPE(KF_MEASURE, st);
  measure_diag_kernel<<<(N + 255) / 256, 256, 0, st>>>(G, N, t, raw);
  DQ_KSCOPE(KF_MEASURE, st);
  measure_finalize_kernel<<<1, 1, 0, st>>>(raw, N, thop, t.wkc != nullptr, obs);
  return cudaGetLastError();
}

}  // namespace dq
