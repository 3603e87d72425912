// Autotuner of the delay rank k and the refresh interval n_stab: every
// candidate pair is measured on a fresh chain of the workload (CUDA events
// on a stream of its own around `sweeps` sweeps after `warmup` untimed
// ones), a pair whose drift |G_wrapped - G_fresh| exceeds the bar is not
// admissible, and the fastest admissible pair wins. The paper fixes both by
// hand; k trades the serial Metropolis block against the rank-k flush, and
// n_stab trades the refresh cost against the drift.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace dq {

// Index of the admissible candidate with the least time (the first in
// candidate order on ties), -1 if none: a time < 0 marks an inadmissible one.
static int autotune_pick(const std::vector<double> &sec) {
  int best = -1;
  for (int i = 0; i < (int)sec.size(); ++i)
    if (sec[i] >= 0.0 && (best < 0 || sec[i] < sec[best])) best = i;
  return best;
}

// One candidate: seconds per timed sweep, or -1 when its drift is above the bar.
static dqmc_status autotune_trial(int L, double beta, double dtau, double U, double mu, uint64_t seed,
                                  int precision, int k, int n_stab, int warmup, int sweeps, double drift_bar,
                                  double *sec) {
  dqmc_ctx *c = nullptr;
  dqmc_status st = dqmc_create(L, beta, dtau, U, mu, seed, &c);
  if (st != DQMC_OK) return st;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto done = [&](dqmc_status r) {
    // the chain first (it synchronises its streams), then the stream it used
    dqmc_destroy(c);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return r;
  };
  const std::string what = "autotune k=" + std::to_string(k) + " n_stab=" + std::to_string(n_stab) + ": ";
  // a drift above the bar disqualifies the pair; only the library's hard
  // limit (a broken chain) ends the trial with an error
  if ((st = dqmc_set_option(c, "k", k)) != DQMC_OK || (st = dqmc_set_option(c, "n_stab", n_stab)) != DQMC_OK ||
      (st = dqmc_set_option(c, "precision", precision)) != DQMC_OK ||
      (st = dqmc_set_option(c, "drift_limit", 10.0)) != DQMC_OK)
    return done(fail(st, what + dqmc_last_error()));
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return done(cuda_fail(e, "autotune stream / events"));
  if ((st = dqmc_set_stream(c, s)) != DQMC_OK) return done(st);
  if (warmup > 0 && (st = dqmc_sweep(c, warmup, 0)) != DQMC_OK) return done(st);
  if ((e = cudaEventRecord(e0, s)) != cudaSuccess) return done(cuda_fail(e, "autotune event"));
  if ((st = dqmc_sweep(c, sweeps, 0)) != DQMC_OK) return done(st);
  if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess)
    return done(cuda_fail(e, "autotune event"));
  float ms = 0.f;
  if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return done(cuda_fail(e, "autotune timing"));
  dqmc_stats stats;
  if ((st = dqmc_get_stats(c, &stats)) != DQMC_OK) return done(st);
  *sec = stats.max_drift <= drift_bar ? ms * 1e-3 / sweeps : -1.0;
  return done(DQMC_OK);
}

}  // namespace dq

extern "C" dqmc_status dqmc_autotune(int L, double beta, double dtau, double U, double mu, uint64_t seed,
                                     int precision, const int *ks, int nk, const int *n_stabs, int ns,
                                     int warmup, int sweeps, double drift_bar, int *k_best, int *n_stab_best,
                                     double *sec_per_sweep, double *times) try {
  using namespace dq;
  if (!ks || !n_stabs || nk < 1 || ns < 1 || !k_best || !n_stab_best || !sec_per_sweep)
    return fail(DQMC_EINVAL, "autotune: need non-empty candidate lists and the three outputs");
  if (warmup < 0 || sweeps < 1 || !(drift_bar > 0.0))
    return fail(DQMC_EINVAL, "autotune: need warmup >= 0, sweeps >= 1 and drift_bar > 0");
  if (precision < 0 || precision > 2) return fail(DQMC_EINVAL, "autotune: precision must be 0, 1 or 2");
  for (int a = 0; a < nk; ++a)
    if (ks[a] < 1) return fail(DQMC_EINVAL, "autotune: delay ranks must be >= 1");
  for (int b = 0; b < ns; ++b)
    if (n_stabs[b] < 1) return fail(DQMC_EINVAL, "autotune: refresh intervals must be >= 1");
  std::vector<double> sec((size_t)nk * ns, -1.0);
  for (int a = 0; a < nk; ++a)
    for (int b = 0; b < ns; ++b) {
      dqmc_status st = autotune_trial(L, beta, dtau, U, mu, seed, precision, ks[a], n_stabs[b], warmup, sweeps,
                                      drift_bar, &sec[(size_t)a * ns + b]);
      if (st != DQMC_OK) return st;
    }
  if (times)
    for (size_t i = 0; i < sec.size(); ++i) times[i] = sec[i];
  const int best = autotune_pick(sec);
  if (best < 0) return fail(DQMC_EINVAL, "autotune: no candidate keeps the drift within the bar");
  *k_best = ks[best / ns];
  *n_stab_best = n_stabs[best % ns];
  *sec_per_sweep = sec[best];
  return DQMC_OK;
}
DQ_API_CATCH
