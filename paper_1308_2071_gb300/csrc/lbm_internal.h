// Internal interface between the C-ABI runtime (lbm_api.cu) and the kernel
// translation units.  Not part of the public boundary.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

enum { PREC_F64 = 0, PREC_F32 = 1, PREC_F16 = 2 };

// Coefficients of one lattice in both arithmetic types.
struct CoefSet {
    Coef<double> d;
    Coef<float> f;
};

struct StepLaunch {
    int precision;
    const void* src;
    void* dst;
    const void* phi;  // per-cell porosity in the storage type, or nullptr
    Geom gm;
    int bx, by;
    int* status;
    cudaStream_t stream;
};

struct ObserveLaunch {
    int precision;
    const void* prev;  // B_{n-1}: pulling from it rebuilds the post-stream state S_n
    const void* phi;
    Geom gm;
    void *ux, *uy, *T, *p;  // optional dense outputs (arithmetic type)
    void* snap;             // velocity snapshot of the previous call (2 per node)
    int snap_valid;
    double* partials;       // 4 * nblocks
    int nblocks;
    double L, dT;
    const int* status;
    double* out;            // 7 doubles
    cudaStream_t stream;
};

struct ReadStateLaunch {
    int precision;
    const void* prev;
    const void* phi;
    Geom gm;
    double *f, *g;
    int nblocks;
    cudaStream_t stream;
};

cudaError_t launch_step(const StepLaunch& L, const CoefSet& cs);
cudaError_t launch_observe(const ObserveLaunch& L, const CoefSet& cs);
cudaError_t launch_nusselt(const ObserveLaunch& L, const CoefSet& cs);
cudaError_t launch_read_state(const ReadStateLaunch& L, const CoefSet& cs);
// Bytes of one state buffer (9 flow + 5 thermal planes) and of a porosity field.
size_t state_buffer_bytes(int precision, int plane);
size_t phi_bytes(int precision, int plane);

cudaError_t launch_convert_phi(const void* in, int in_is_double, void* out, int precision, const Geom& gm,
                               int nblocks, cudaStream_t s);

}  // namespace lbm
