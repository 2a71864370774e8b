// Input-wave estimate and misfit ERR on the GPU (Section 2, Eq. (2)).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace gsw {

constexpr int kMisfitMaxUnknowns = 384;  // 3 * n_shifts

struct MisfitWork {
  double* buf = nullptr;  // device scratch (grown on demand)
  size_t bytes = 0;
  double* host = nullptr;  // pinned results
};

// Returns 0 on success, 1 CUDA error (*ce set), 2 allocation failure,
// 3 invalid input (msg set).
int misfit_run(MisfitWork& w, cudaStream_t s, int n_rec, int n_t, const double* G, const double* obs,
               int stride, int n_shifts, double tau, double* err, double* c_out, char* msg,
               size_t msg_len, cudaError_t* ce);
void misfit_free(MisfitWork& w, cudaStream_t s);

// Allocation-free variant: device inputs and outputs, working memory in a
// fixed file-scope __device__ array.
constexpr int kNoAllocMaxShifts = 64;
constexpr int kNoAllocMaxRec = 1024;
int misfit_run_noalloc(cudaStream_t s, int device, int n_rec, int n_t, const double* G_dev, const double* obs_dev,
                       int stride, int n_shifts, double tau, double* err_dev, double* c_dev, char* msg,
                       size_t msg_len, cudaError_t* ce);

}  // namespace gsw
