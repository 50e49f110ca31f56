// Compute entry points: kldi_density, kldi_vxc, kldi_exc, kldi_exc_batched.
// Every step runs in this library's CUDA kernels on the plan's stream.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

using namespace kldi;

namespace kldi {
kldi_status ensure_tile_buffers(kldi_plan* P, int prec);

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace kldi

using kldi::is_device_ptr;

namespace {

// Stage names of the NVTX ranges that bracket each stage's launches (a
// profiler can filter kernels by them, e.g. ncu --nvtx --nvtx-include).
const char* const kStageNames[] = {"kldi:dprep", "kldi:phi", "kldi:rho", "kldi:xc", "kldi:x", "kldi:v", "kldi:finish"};

// Stage timing: record an event pair around `fn` when profiling is on.
template <typename F>
kldi_status staged(kldi_plan* P, int stage, int launches, F&& fn) {
  P->launch_count += launches;
  struct Range {
    explicit Range(int s) { nvtxRangePushA(kStageNames[s]); }
    ~Range() { nvtxRangePop(); }
  } range(stage);
  if (!P->prof || P->prof_stage.size() * 2 + 2 > P->prof_ev.size()) return fn();
  const size_t k = P->prof_stage.size() * 2;
  KLDI_TRY_CUDA(cudaEventRecord(P->prof_ev[k], P->stream));
  KLDI_TRY(fn());
  KLDI_TRY_CUDA(cudaEventRecord(P->prof_ev[k + 1], P->stream));
  P->prof_stage.push_back(stage);
  P->prof_launches.push_back(launches);
  return KLDI_OK;
}


// D -> per-evaluation operands (block maxima; split tiles for tensor modes).
kldi_status prepare_D(kldi_plan* P, const double* D) {
  return staged(P, KLDI_STAGE_DPREP, P->prec == KLDI_FP64 ? 1 : 3, [&]() -> kldi_status {
    KLDI_TRY(launch_dmax(P, D, P->stream));
    if (P->prec != KLDI_FP64) KLDI_TRY(launch_dsplit(P, D, P->stream));
    return KLDI_OK;
  });
}

kldi_status density_batch(kldi_plan* P, const Batch& b, const double* D, double* rho, double* grad) {
  if (P->prec == KLDI_FP64) {
    KLDI_TRY(staged(P, KLDI_STAGE_PHI, 1, [&] { return launch_phi64(P, b, P->stream); }));
    KLDI_TRY(staged(P, KLDI_STAGE_RHO, 1, [&] { return launch_rho64(P, b, D, rho, grad, P->stream); }));
  } else {
    KLDI_TRY(staged(P, KLDI_STAGE_PHI, 1, [&] { return launch_phi_split(P, b, P->stream); }));
    KLDI_TRY(staged(P, KLDI_STAGE_RHO, 1, [&] { return launch_rho_tc(P, b, rho, grad, P->stream); }));
  }
  return KLDI_OK;
}

kldi_status potential_batch(kldi_plan* P, const Batch& b, int xc, const double* rho, const double* grad,
                            double* V, bool phi_ready) {
  KLDI_TRY(staged(P, KLDI_STAGE_XC, 1, [&] { return launch_xc(P, b, xc, rho, grad, P->stream); }));
  if (P->prec == KLDI_FP64) {
    if (!phi_ready) KLDI_TRY(staged(P, KLDI_STAGE_PHI, 1, [&] { return launch_phi64(P, b, P->stream); }));
    KLDI_TRY(staged(P, KLDI_STAGE_X, 1, [&] { return launch_x64(P, b, P->stream); }));
    KLDI_TRY(staged(P, KLDI_STAGE_V, 1, [&] { return launch_v64(P, b, V, P->stream); }));
  } else {
    // the V product's operands come from the X kernel; the per-point Phi slices are not
    // needed, but BF16X10's X kernel reads the radial factors the Phi kernel writes
    if (!phi_ready && P->prec == KLDI_BF16X10)
      KLDI_TRY(staged(P, KLDI_STAGE_PHI, 1, [&] { return launch_phi_split(P, b, P->stream); }));
    KLDI_TRY(staged(P, KLDI_STAGE_X, 1, [&] { return launch_x_split(P, b, P->stream); }));
    KLDI_TRY(staged(P, KLDI_STAGE_V, 1, [&] { return launch_v_tc(P, b, V, P->stream); }));
  }
  return KLDI_OK;
}

// After a synchronising call: report a bounded device wait that gave up.
kldi_status check_device_error(kldi_plan* P) {
  int e = 0;
  KLDI_TRY_CUDA(cudaMemcpy(&e, P->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) {
    cudaMemset(P->d_err, 0, sizeof(int));
    set_error("a device-side bounded wait gave up (code %d)", e);
    return e == 101 ? KLDI_EUNSUPPORTED : KLDI_ETIMEOUT;
  }
  return KLDI_OK;
}

kldi_status check_xc(const kldi_plan* P, int xc) {
  if (xc < KLDI_XC_LDA_X || xc > KLDI_XC_MLP) {
    set_error("functional %d is not available in this call", xc);
    return KLDI_EINVAL;
  }
  if (xc != KLDI_XC_LDA_X && !P->gga) {
    set_error("a GGA functional needs a plan screened with a GGA functional (basis gradients)");
    return KLDI_EINVAL;
  }
  if (xc == KLDI_XC_MLP && !P->mlp) {
    set_error("KLDI_XC_MLP needs a network attached with kldi_plan_set_mlp");
    return KLDI_EINVAL;
  }
  return KLDI_OK;
}

// D in the caller's function order (device) -> the plan's order.
kldi_status internal_D(kldi_plan* P, const double*& D) {
  if (!P->d_fnperm) return KLDI_OK;
  const double* src = D;
  KLDI_TRY(staged(P, KLDI_STAGE_DPREP, 1, [&] { return launch_permute(P, src, P->d_Dint, true, P->stream); }));
  D = P->d_Dint;
  return KLDI_OK;
}

kldi_status exc_device(kldi_plan* P, int xc, const double* D, double* V, double* exc) {
  if (P->d_fnperm) {
    // reordered plan: evaluate in the internal order, then V to the caller's order
    KLDI_TRY(internal_D(P, D));
    double* Vc = V;
    V = P->d_Vint;
    KLDI_TRY(ensure_tile_buffers(P, P->prec));
    KLDI_TRY(prepare_D(P, D));
    KLDI_TRY_CUDA(cudaMemsetAsync(V, 0, sizeof(double) * P->nbf * P->nbf, P->stream));
    for (const Batch& b : P->batches) {
      KLDI_TRY(density_batch(P, b, D, P->d_rho, P->d_grad));
      KLDI_TRY(potential_batch(P, b, xc, P->d_rho, P->d_grad, V, true));
    }
    KLDI_TRY(staged(P, KLDI_STAGE_FINISH, 3, [&]() -> kldi_status {
      KLDI_TRY(launch_finish(P, V, exc, P->stream));
      return launch_permute(P, V, Vc, false, P->stream);
    }));
    return KLDI_OK;
  }
  KLDI_TRY(ensure_tile_buffers(P, P->prec));
  KLDI_TRY(prepare_D(P, D));
  KLDI_TRY_CUDA(cudaMemsetAsync(V, 0, sizeof(double) * P->nbf * P->nbf, P->stream));
  for (const Batch& b : P->batches) {
    KLDI_TRY(density_batch(P, b, D, P->d_rho, P->d_grad));
    KLDI_TRY(potential_batch(P, b, xc, P->d_rho, P->d_grad, V, true));
  }
  KLDI_TRY(staged(P, KLDI_STAGE_FINISH, 2, [&] { return launch_finish(P, V, exc, P->stream); }));
  return KLDI_OK;
}

}  // namespace

extern "C" kldi_status kldi_density(kldi_plan* P, const double* D, double* rho, double* grad) {
  return kldi::guarded("kldi_density", [&]() -> kldi_status {
    if (!P || !D || !rho) { set_error("kldi_density: null argument"); return KLDI_EINVAL; }
    if (P->gga && !grad) { set_error("kldi_density: a GGA plan needs grad"); return KLDI_EINVAL; }
    const bool host_out = !is_device_ptr(rho);
    if (P->gga && is_device_ptr(grad) == host_out) {
      // checked before any work: the kernels write rho and grad where they point
      set_error("kldi_density: rho and grad must both be device or both host memory");
      return KLDI_EINVAL;
    }
    const size_t nbf2 = (size_t)P->nbf * P->nbf;
    const double* dD = D;
    if (!is_device_ptr(D)) {
      KLDI_TRY_CUDA(cudaMemcpyAsync(P->d_D, D, nbf2 * 8, cudaMemcpyHostToDevice, P->stream));
      dD = P->d_D;
    }
    double* drho = host_out ? P->d_rho : rho;
    double* dgrad = P->gga ? (host_out ? P->d_grad : grad) : P->d_grad;
    KLDI_TRY(ensure_tile_buffers(P, P->prec));
    KLDI_TRY(internal_D(P, dD));
    KLDI_TRY(prepare_D(P, dD));
    for (const Batch& b : P->batches) KLDI_TRY(density_batch(P, b, dD, drho, dgrad));
    if (host_out) {
      KLDI_TRY_CUDA(cudaMemcpyAsync(rho, drho, P->npoints * 8, cudaMemcpyDeviceToHost, P->stream));
      if (P->gga) KLDI_TRY_CUDA(cudaMemcpyAsync(grad, dgrad, P->npoints * 24, cudaMemcpyDeviceToHost, P->stream));
      KLDI_TRY_CUDA(cudaStreamSynchronize(P->stream));
      KLDI_TRY(check_device_error(P));
    }
    KLDI_TRY_CUDA(cudaGetLastError());
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_vxc(kldi_plan* P, int xc, const double* rho, const double* grad, double* V,
                                double* Exc) {
  return kldi::guarded("kldi_vxc", [&]() -> kldi_status {
    if (!P || !rho || !V || !Exc) { set_error("kldi_vxc: null argument"); return KLDI_EINVAL; }
    KLDI_TRY(check_xc(P, xc));
    if (xc != KLDI_XC_LDA_X && !grad) { set_error("kldi_vxc: the GGA needs grad"); return KLDI_EINVAL; }
    KLDI_TRY(ensure_tile_buffers(P, P->prec));
    const double* drho = rho;
    const double* dgrad = grad;
    if (!is_device_ptr(rho)) {
      KLDI_TRY_CUDA(cudaMemcpyAsync(P->d_rho, rho, P->npoints * 8, cudaMemcpyHostToDevice, P->stream));
      drho = P->d_rho;
    }
    if (grad && !is_device_ptr(grad)) {
      KLDI_TRY_CUDA(cudaMemcpyAsync(P->d_grad, grad, P->npoints * 24, cudaMemcpyHostToDevice, P->stream));
      dgrad = P->d_grad;
    }
    if (!dgrad) dgrad = P->d_grad;
    const bool hostV = !is_device_ptr(V), hostE = !is_device_ptr(Exc);
    double* dV = hostV ? P->d_V : V;
    double* dE = hostE ? P->d_exc : Exc;
    double* dVc = dV;
    if (P->d_fnperm) dV = P->d_Vint;   // reordered plan: V to the caller's order at the end
    KLDI_TRY_CUDA(cudaMemsetAsync(dV, 0, sizeof(double) * P->nbf * P->nbf, P->stream));
    for (const Batch& b : P->batches) KLDI_TRY(potential_batch(P, b, xc, drho, dgrad, dV, false));
    KLDI_TRY(staged(P, KLDI_STAGE_FINISH, 2, [&] { return launch_finish(P, dV, dE, P->stream); }));
    if (P->d_fnperm) {
      KLDI_TRY(staged(P, KLDI_STAGE_FINISH, 1, [&] { return launch_permute(P, dV, dVc, false, P->stream); }));
      dV = dVc;
    }
    if (hostV) KLDI_TRY_CUDA(cudaMemcpyAsync(V, dV, sizeof(double) * P->nbf * P->nbf, cudaMemcpyDeviceToHost, P->stream));
    if (hostE) KLDI_TRY_CUDA(cudaMemcpyAsync(Exc, dE, 8, cudaMemcpyDeviceToHost, P->stream));
    if (hostV || hostE) {
      KLDI_TRY_CUDA(cudaStreamSynchronize(P->stream));
      KLDI_TRY(check_device_error(P));
    }
    KLDI_TRY_CUDA(cudaGetLastError());
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_exc(kldi_plan* P, int xc, const double* D, double* V, double* Exc) {
  return kldi::guarded("kldi_exc", [&]() -> kldi_status {
    if (!P || !D || !V || !Exc) { set_error("kldi_exc: null argument"); return KLDI_EINVAL; }
    KLDI_TRY(check_xc(P, xc));
    const size_t nbf2 = (size_t)P->nbf * P->nbf;
    const double* dD = D;
    if (!is_device_ptr(D)) {
      KLDI_TRY_CUDA(cudaMemcpyAsync(P->d_D, D, nbf2 * 8, cudaMemcpyHostToDevice, P->stream));
      dD = P->d_D;
    }
    const bool hostV = !is_device_ptr(V), hostE = !is_device_ptr(Exc);
    double* dV = hostV ? P->d_V : V;
    double* dE = hostE ? P->d_exc : Exc;
    KLDI_TRY(exc_device(P, xc, dD, dV, dE));
    if (hostV) KLDI_TRY_CUDA(cudaMemcpyAsync(V, dV, nbf2 * 8, cudaMemcpyDeviceToHost, P->stream));
    if (hostE) KLDI_TRY_CUDA(cudaMemcpyAsync(Exc, dE, 8, cudaMemcpyDeviceToHost, P->stream));
    if (hostV || hostE) {
      KLDI_TRY_CUDA(cudaStreamSynchronize(P->stream));
      KLDI_TRY(check_device_error(P));
    }
    KLDI_TRY_CUDA(cudaGetLastError());
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_exc_grad(kldi_plan* P, int xc, const double* D, double* G, double* Exc) {
  return kldi::guarded("kldi_exc_grad", [&]() -> kldi_status {
    if (!P || !D || !G || !Exc) { set_error("kldi_exc_grad: null argument"); return KLDI_EINVAL; }
    KLDI_TRY(check_xc(P, xc));
    if (P->prec != KLDI_FP64 && !P->rec_fit_all) {
      set_error("kldi_exc_grad: a basis block has more than 40 shells or 80 primitives (tensor-core gradient)");
      return KLDI_EUNSUPPORTED;
    }
    const size_t nbf2 = (size_t)P->nbf * P->nbf;
    const double* dD = D;
    if (!is_device_ptr(D)) {
      KLDI_TRY_CUDA(cudaMemcpyAsync(P->d_D, D, nbf2 * 8, cudaMemcpyHostToDevice, P->stream));
      dD = P->d_D;
    }
    // G and Exc may be host or device memory independently of each other
    const bool hostG = !is_device_ptr(G), hostE = !is_device_ptr(Exc);
    if (!P->d_G) {
      KLDI_TRY_CUDA(cudaMalloc(&P->d_G, sizeof(double) * 3 * std::max(P->natm, 1)));
    }
    double* dG = hostG ? P->d_G : G;
    double* dE = hostE ? P->d_exc : Exc;
    KLDI_TRY(ensure_tile_buffers(P, P->prec));
    if (P->prec != KLDI_FP64 && !P->d_zscale) {
      KLDI_TRY_CUDA(cudaMalloc(&P->d_zscale, sizeof(float) * std::max<int64_t>(P->npoints, 1)));
    }
    KLDI_TRY(internal_D(P, dD));
    KLDI_TRY(prepare_D(P, dD));
    KLDI_TRY_CUDA(cudaMemsetAsync(dG, 0, sizeof(double) * 3 * P->natm, P->stream));
    for (const Batch& b : P->batches) {
      KLDI_TRY(density_batch(P, b, dD, P->d_rho, P->d_grad));
      KLDI_TRY(staged(P, KLDI_STAGE_XC, 1, [&] { return launch_xc(P, b, xc, P->d_rho, P->d_grad, P->stream); }));
      if (P->prec == KLDI_FP64) {
        KLDI_TRY(staged(P, KLDI_STAGE_X, 1, [&] { return launch_x64(P, b, P->stream); }));
        KLDI_TRY(staged(P, KLDI_STAGE_V, 1, [&] { return launch_grad64(P, b, dD, dG, P->stream); }));
      } else {
        // Z tiles (X stage), then the Q and R terms through the density-product kernel (V stage)
        const bool gga_xc = xc != KLDI_XC_LDA_X;
        KLDI_TRY(staged(P, KLDI_STAGE_V, gga_xc ? 3 : 2,
                        [&] { return launch_grad_tc(P, b, gga_xc, dG, P->stream); }));
      }
    }
    KLDI_TRY(staged(P, KLDI_STAGE_FINISH, 1, [&] { return launch_finish(P, nullptr, dE, P->stream); }));
    if (hostG) KLDI_TRY_CUDA(cudaMemcpyAsync(G, dG, sizeof(double) * 3 * P->natm, cudaMemcpyDeviceToHost, P->stream));
    if (hostE) KLDI_TRY_CUDA(cudaMemcpyAsync(Exc, dE, 8, cudaMemcpyDeviceToHost, P->stream));
    if (hostG || hostE) {
      KLDI_TRY_CUDA(cudaStreamSynchronize(P->stream));
      KLDI_TRY(check_device_error(P));
    }
    KLDI_TRY_CUDA(cudaGetLastError());
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_exc_batched(kldi_plan* const* plans, int nframes, int xc, const double* const* D,
                                        double* const* V, double* Exc) {
  return kldi::guarded("kldi_exc_batched", [&]() -> kldi_status {
    if (!plans || nframes <= 0 || !D || !V || !Exc) { set_error("kldi_exc_batched: bad argument"); return KLDI_EINVAL; }
    for (int k = 0; k < nframes; ++k) {
      if (!plans[k] || !D[k] || !V[k]) { set_error("kldi_exc_batched: null entry %d", k); return KLDI_EINVAL; }
      if (!is_device_ptr(D[k]) || !is_device_ptr(V[k])) {
        set_error("kldi_exc_batched: device pointers only (entry %d)", k);
        return KLDI_EINVAL;
      }
      KLDI_TRY(check_xc(plans[k], xc));
    }
    if (!is_device_ptr(Exc)) { set_error("kldi_exc_batched: Exc must be device memory"); return KLDI_EINVAL; }
    // one graph of all frames, launched once on the first plan's stream
    kldi_batch* B = nullptr;
    KLDI_TRY(kldi_batch_create(plans, nframes, xc, D, V, Exc, plans[0]->stream, &B));
    const kldi_status st = kldi_batch_launch(B);
    const kldi_status st2 = kldi_batch_sync(B);
    kldi_batch_free(B);
    KLDI_TRY(st);
    return st2;
  });
}

extern "C" kldi_status kldi_plan_profile(kldi_plan* P, int enable) {
  return kldi::guarded("kldi_plan_profile", [&]() -> kldi_status {
    if (!P) { set_error("kldi_plan_profile: null plan"); return KLDI_EINVAL; }
    if (enable && P->prof_ev.empty()) {
      P->prof_ev.resize(8192);
      for (auto& e : P->prof_ev) KLDI_TRY_CUDA(cudaEventCreate(&e));
    }
    KLDI_TRY_CUDA(cudaStreamSynchronize(P->stream));
    P->prof_stage.clear();
    P->prof_launches.clear();
    P->prof = enable != 0;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_plan_stage_times(kldi_plan* P, double* ms, int64_t* launches) {
  return kldi::guarded("kldi_plan_stage_times", [&]() -> kldi_status {
    if (!P) { set_error("kldi_plan_stage_times: null plan"); return KLDI_EINVAL; }
    KLDI_TRY_CUDA(cudaStreamSynchronize(P->stream));
    double t[KLDI_NSTAGES] = {0};
    int64_t n[KLDI_NSTAGES] = {0};
    for (size_t k = 0; k < P->prof_stage.size(); ++k) {
      float e = 0.f;
      KLDI_TRY_CUDA(cudaEventElapsedTime(&e, P->prof_ev[2 * k], P->prof_ev[2 * k + 1]));
      t[P->prof_stage[k]] += e;
      n[P->prof_stage[k]] += P->prof_launches[k];
    }
    for (int s = 0; s < KLDI_NSTAGES; ++s) {
      if (ms) ms[s] = t[s];
      if (launches) launches[s] = n[s];
    }
    return KLDI_OK;
  });
}

// ---------------------------------------------------------------------------
// Tuning and batched frames.
struct kldi_batch {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<kldi_plan*> plans;
};

// Times `reps` evaluations with tuning t (after one untimed one); ms per evaluation.
static kldi_status time_tuning(kldi_plan* P, int xc, const double* D, int reps, const kldi_tuning& t,
                               cudaEvent_t e0, cudaEvent_t e1, double* ms_out) {
  KLDI_TRY(kldi_plan_set_tuning(P, &t));
  KLDI_TRY(exc_device(P, xc, D, P->d_V, P->d_exc));
  KLDI_TRY_CUDA(cudaEventRecord(e0, P->stream));
  for (int r = 0; r < reps; ++r) KLDI_TRY(exc_device(P, xc, D, P->d_V, P->d_exc));
  KLDI_TRY_CUDA(cudaEventRecord(e1, P->stream));
  KLDI_TRY_CUDA(cudaEventSynchronize(e1));
  KLDI_TRY(check_device_error(P));
  float ms = 0.f;
  KLDI_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  *ms_out = ms / reps;
  return KLDI_OK;
}

extern "C" kldi_status kldi_plan_autotune(kldi_plan* P, int xc, const double* D, int reps, kldi_tuning* best,
                                          double* best_ms) {
  return kldi::guarded("kldi_plan_autotune", [&]() -> kldi_status {
    if (!P || !D || reps < 1 || !is_device_ptr(D)) {
      set_error("kldi_plan_autotune: bad argument (D must be device memory, reps >= 1)");
      return KLDI_EINVAL;
    }
    KLDI_TRY(check_xc(P, xc));
    cudaEvent_t e0, e1;
    KLDI_TRY_CUDA(cudaEventCreate(&e0));
    KLDI_TRY_CUDA(cudaEventCreate(&e1));
    const int prof = P->prof;
    P->prof = 0;
    // coordinate search: the density product's N tile at the default V
    // decomposition, then the V window alignment, then the V work-item span
    // with the chosen tile and alignment
    kldi_tuning bt{0, 0, 0};
    double bms = 1e300;
    kldi_status st = KLDI_OK;
    std::vector<int> tiles = {0};
    if (P->prec == KLDI_BF16X3 || P->prec == KLDI_BF16X6) tiles = {128, 64};
    for (int nt : tiles) {
      double ms = 0.0;
      const kldi_tuning t{0, nt, 0};
      if ((st = time_tuning(P, xc, D, reps, t, e0, e1, &ms)) != KLDI_OK) break;
      if (ms < bms) { bms = ms; bt = t; }
    }
    const int aligns[] = {4, 1};
    for (int k = 0; k < 2 && st == KLDI_OK && P->prec != KLDI_FP64; ++k) {
      double ms = 0.0;
      const kldi_tuning t{0, bt.rho_ntile, aligns[k]};
      if ((st = time_tuning(P, xc, D, reps, t, e0, e1, &ms)) != KLDI_OK) break;
      if (ms < bms) { bms = ms; bt = t; }
    }
    const int segs[] = {16, 32, 128, 256};
    for (int k = 0; k < 4 && st == KLDI_OK && P->prec != KLDI_FP64; ++k) {
      double ms = 0.0;
      const kldi_tuning t{segs[k], bt.rho_ntile, bt.v_align};
      if ((st = time_tuning(P, xc, D, reps, t, e0, e1, &ms)) != KLDI_OK) break;
      if (ms < bms) { bms = ms; bt = t; }
    }
    P->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    KLDI_TRY(st);
    KLDI_TRY(kldi_plan_set_tuning(P, &bt));
    if (best) *best = bt;
    if (best_ms) *best_ms = bms;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_batch_create(kldi_plan* const* plans, int nframes, int xc, const double* const* D,
                                         double* const* V, double* Exc, void* stream, kldi_batch** out) {
  return kldi::guarded("kldi_batch_create", [&]() -> kldi_status {
    if (!plans || nframes <= 0 || !D || !V || !Exc || !out) {
      set_error("kldi_batch_create: bad argument");
      return KLDI_EINVAL;
    }
    *out = nullptr;
    if (!is_device_ptr(Exc)) { set_error("kldi_batch_create: Exc must be device memory"); return KLDI_EINVAL; }
    for (int k = 0; k < nframes; ++k) {
      if (!plans[k] || !D[k] || !V[k]) { set_error("kldi_batch_create: null entry %d", k); return KLDI_EINVAL; }
      if (!is_device_ptr(D[k]) || !is_device_ptr(V[k])) {
        set_error("kldi_batch_create: device pointers only (entry %d)", k);
        return KLDI_EINVAL;
      }
      if (plans[k]->device != plans[0]->device) {
        set_error("kldi_batch_create: plans on different devices");
        return KLDI_EINVAL;
      }
      KLDI_TRY(check_xc(plans[k], xc));
      KLDI_TRY(ensure_tile_buffers(plans[k], plans[k]->prec));
    }
    KLDI_TRY(prepare_tc_kernels());
    kldi_batch* B = new kldi_batch;
    B->plans.assign(plans, plans + nframes);
    B->stream = static_cast<cudaStream_t>(stream);
    if (!B->stream) {
      if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete B;
        set_error("kldi_batch_create: stream creation failed");
        return KLDI_ECUDA;
      }
      B->own_stream = true;
    }
    for (kldi_plan* P : B->plans) cudaStreamSynchronize(P->stream);
    if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      set_error("kldi_batch_create: %s", cudaGetErrorString(cudaGetLastError()));
      kldi_batch_free(B);
      return KLDI_ECUDA;
    }
    kldi_status st = KLDI_OK;
    for (int k = 0; k < nframes && st == KLDI_OK; ++k) {
      kldi_plan* P = plans[k];
      const cudaStream_t keep = P->stream;
      const int prof = P->prof;
      P->stream = B->stream;
      P->prof = 0;
      st = exc_device(P, xc, D[k], V[k], Exc + k);
      P->stream = keep;
      P->prof = prof;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(B->stream, &graph);
    if (st == KLDI_OK && (ec != cudaSuccess || !graph)) {
      set_error("kldi_batch_create: capture failed: %s", cudaGetErrorString(ec));
      st = KLDI_ECUDA;
    }
    if (st == KLDI_OK && cudaGraphInstantiate(&B->exec, graph, 0) != cudaSuccess) {
      set_error("kldi_batch_create: graph instantiation failed: %s", cudaGetErrorString(cudaGetLastError()));
      st = KLDI_ECUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (st != KLDI_OK) {
      kldi_batch_free(B);
      return st;
    }
    *out = B;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_batch_launch(kldi_batch* B) {
  return kldi::guarded("kldi_batch_launch", [&]() -> kldi_status {
    if (!B || !B->exec) { set_error("kldi_batch_launch: null batch"); return KLDI_EINVAL; }
    KLDI_TRY_CUDA(cudaGraphLaunch(B->exec, B->stream));
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_batch_sync(kldi_batch* B) {
  return kldi::guarded("kldi_batch_sync", [&]() -> kldi_status {
    if (!B) { set_error("kldi_batch_sync: null batch"); return KLDI_EINVAL; }
    KLDI_TRY_CUDA(cudaStreamSynchronize(B->stream));
    for (kldi_plan* P : B->plans) KLDI_TRY(check_device_error(P));
    return KLDI_OK;
  });
}

extern "C" void kldi_batch_free(kldi_batch* B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
}
