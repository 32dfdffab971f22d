// FFT tile autotuner and batched multi-plan solve.
//
// The column kernel's transforms split each length-nz pencil over T lanes of a warp;
// T trades shuffle and twiddle work against registers and shared memory.
// psfd_autotune times every compiled T for the plan's shape with CUDA events and
// keeps the fastest; results are cached per (nx, ny, nz, nrhs) for the process.
//
// psfd_solve_batched runs many independent solves (masks of different size,
// angles, polarisations) concurrently: a pool of host workers takes plans in
// order and runs psfd_solve_ex on each plan's own stream, so small problems fill
// the GPU together.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "internal.h"

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune;
}  // namespace

extern "C" int psfd_autotune(psfd_plan P, int* chosen_T) {
  if (!P) { psfd_set_error("psfd_autotune: null plan"); return PSFD_ERR_ARG; }
  if (!P->have_background) { psfd_set_error("psfd_autotune: call psfd_background first"); return PSFD_ERR_STATE; }
  const auto key = std::make_tuple(P->nx, P->ny, P->nz, P->nrhs);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      P->axial_T = it->second;
      if (chosen_T) *chosen_T = it->second;
      return PSFD_OK;
    }
  }
  int cand[4];
  const int nc = axial_candidates(P->nz, cand);
  cudaEvent_t e0, e1;
  PSFD_CUDA_TRY(cudaEventCreate(&e0));
  PSFD_CUDA_TRY(cudaEventCreate(&e1));
  PSFD_CUDA_TRY(cudaMemsetAsync(P->tmpA, 0, (size_t)P->nrhs * P->nvec * sizeof(cf), P->stream));
  float best = 1e30f;
  int bestT = cand[0];
  for (int i = 0; i < nc; ++i) {
    P->axial_T = cand[i];
    int rc = launch_axial(P, P->tmpA, P->tmpB, 0, nullptr, P->nrhs);   // warm-up
    if (rc) return rc;
    PSFD_CUDA_TRY(cudaEventRecord(e0, P->stream));
    for (int k = 0; k < 5; ++k)
      if ((rc = launch_axial(P, P->tmpA, P->tmpB, 0, nullptr, P->nrhs))) return rc;
    PSFD_CUDA_TRY(cudaEventRecord(e1, P->stream));
    PSFD_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    PSFD_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) { best = ms; bestT = cand[i]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->axial_T = bestT;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = bestT;
  }
  if (chosen_T) *chosen_T = bestT;
  return PSFD_OK;
}

extern "C" int psfd_solve_batched(const psfd_plan* plans, int nplans, const psfd_c64* const* b,
                                  const psfd_c64* const* x0, psfd_c64* const* E, const psfd_solve_opts_t* opts,
                                  psfd_info_t* info, int nworkers) {
  if (!plans || nplans <= 0 || !b || !E || !opts || !info) {
    psfd_set_error("psfd_solve_batched: null argument");
    return PSFD_ERR_ARG;
  }
  std::vector<long> off(nplans + 1, 0);
  for (int i = 0; i < nplans; ++i) {
    if (!plans[i] || !b[i] || !E[i]) { psfd_set_error("psfd_solve_batched: null entry %d", i); return PSFD_ERR_ARG; }
    off[i + 1] = off[i] + plans[i]->nrhs;
  }
  int dev = 0;
  PSFD_CUDA_TRY(cudaGetDevice(&dev));
  const int nw = std::max(1, std::min(nworkers > 0 ? nworkers : 8, nplans));
  std::atomic<int> next{0};
  std::vector<int> rcs(nplans, PSFD_OK);
  std::vector<std::string> msgs(nplans);   // a worker's error text (the error string is per thread)
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= nplans) break;
      rcs[i] = psfd_solve_ex(plans[i], b[i], x0 ? x0[i] : nullptr, E[i], opts, info + off[i], nullptr, 0);
      if (rcs[i] != PSFD_OK) msgs[i] = psfd_last_error();
    }
  };
  std::vector<std::thread> pool;
  for (int k = 0; k < nw; ++k) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  int worst = PSFD_OK;
  for (int i = 0; i < nplans; ++i) {
    if (rcs[i] == PSFD_ERR_ARG || rcs[i] == PSFD_ERR_CUDA || rcs[i] == PSFD_ERR_STATE) {
      psfd_set_error("psfd_solve_batched: plan %d: %s", i, msgs[i].c_str());
      return rcs[i];
    }
    if (rcs[i] != PSFD_OK && worst == PSFD_OK) worst = rcs[i];
  }
  return worst;
}
