// Input-wave estimate and misfit ERR on the GPU (Section 2, Eq. (2)).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace gsw {

constexpr int kMisfitMaxUnknowns = 384;  // 3 * n_shifts

// Device scratch of the misfit, from the context's allocator (alloc(bytes,
// stream, user) / free_(ptr, stream, user); cudaMallocAsync when unset).
struct MisfitWork {
  double* buf = nullptr;  // device scratch (grown on demand)
  size_t bytes = 0;
  double* host = nullptr;  // pinned results
  void* (*alloc)(size_t, void*, void*) = nullptr;
  void (*free_)(void*, void*, void*) = nullptr;
  void* user = nullptr;
};

// Returns 0 on success, 1 CUDA error (*ce set), 2 allocation failure,
// 3 invalid input (msg set).  G and obs are host arrays.
int misfit_run(MisfitWork& w, cudaStream_t s, int n_rec, int n_t, const double* G, const double* obs,
               int stride, int n_shifts, double tau, double* err, double* c_out, char* msg,
               size_t msg_len, cudaError_t* ce);
// Same, with the Green's functions gathered on the device from the receiver
// histories of the three input directions: wave[j] [n_rec][3][n_steps] (the
// first n_t samples are used); obs is a host array.
int misfit_run_waves(MisfitWork& w, cudaStream_t s, int n_rec, int n_t, int n_steps, const double* const wave[3],
                     const double* obs, int stride, int n_shifts, double tau, double* err, double* c_out, char* msg,
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
