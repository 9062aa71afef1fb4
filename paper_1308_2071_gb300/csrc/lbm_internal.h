// Internal interface between the C-ABI runtime (lbm_api.cu) and the kernel
// translation units.  Not part of the public boundary.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {

// Names one call of the C-ABI in a profiler's timeline (an NVTX range for the
// call's duration on the host); costs next to nothing when no profiler is
// attached.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Lattice parameters derived from lbm_params (Section 4 set-up).
struct Derived {
    double L, tau_nu, tau_T, nu, gbeta, K, Fphi, T0, dT, Q;
};

// Validates p and fills the derived parameters, the coefficients in both
// arithmetic types and the geometry; returns LBM_OK or LBM_ERR_ARG with *why.
int setup_lattice(const lbm_params* p, Derived* dv, struct CoefSet* cs, Geom* gm, std::string* why);

// Header of a checkpoint (lbm_save / lbm_load); the payload that follows is
// B_{n-1} (version 2), or B_{n-1} then B_n (version 1, still read).
struct CkptHeader {
    char magic[8];
    int version, nx, ny, precision;
    long t;
    long payload;
};

// Version 3 stores LBM_F32 and LBM_F32_STORE_F16 lattices with their 8-bit
// temperature frames; the FP64 and FP32-framed layouts are those of versions
// 1 and 2, which stay readable.
inline bool ckpt_layout_current(int version, int precision) {
    return version == 3 || precision == LBM_F64 || precision == LBM_F32_FRAMED;
}

// Bounds-checked build: device address of the out-of-plane access counter
// (nullptr in the normal build).
int* oob_counter();

// Error text returned by lbm_last_error(NULL) (calls without a handle).
void set_global_error(const std::string& msg);

constexpr int kReduceBlocks = 1216;  // 152 SMs x 8; fixed so FP64 sums are reproducible

enum { PREC_F64 = 0, PREC_F32 = 1, PREC_F16 = 2, PREC_F32T = 3 };

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
    int npt = 1;  // nodes per thread: 1, 2 (along y) or 3 (two along x)
    int* status;
    cudaStream_t stream;
    bool pdl = false;  // launch as a programmatic dependent of the previous step
    double* obs = nullptr;  // observing step: wall-column temperatures (kObsCols per row)
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
    unsigned* counter = nullptr;  // launch_nusselt: zero-initialised block counter
    const double* obs = nullptr;  // launch_nusselt: read the wall columns an observing step stored
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
// One reverse sweep of the discrete adjoint (lbm_adjoint.cu).  ckpt holds the
// states B_{sK-1} for every segment s (slot 0: the rest state), seg has room
// for 2 (K - 1) recomputed states (two segments), madj for two adjoint
// lattices (14 planes in the arithmetic type), gphi one double per node.
struct AdjointJob {
    int precision;
    Geom gm;
    const void* coef;  // Coef<R> of the arithmetic type
    long nsteps, ckpt_every;
    size_t buf_bytes;
    const void* ckpt;
    void* seg;
    void* madj;
    double* gphi;
    const void* phi;
    int* status;
    double L, dT;
    void* out;  // ny*nx dense, double (FP64) or float (FP32)
    int bx = 128, by = 2, npt = 1;  // launch shape of the recomputing forward steps
    cudaStream_t stream;
};
cudaError_t launch_adjoint_sweep(const AdjointJob& J);

struct SteadyCheckLaunch {
    int precision;
    const void* prev;
    Geom gm;
    double L, dT;
    const int* status;
    double tol;
    long max_checks;
    double* state;  // 8 doubles
    cudaGraphConditionalHandle cond;
    cudaStream_t stream;
};
cudaError_t launch_steady_check(const SteadyCheckLaunch& L, const CoefSet& cs);
// out: 3 doubles per column (max T, min psi, max psi)
cudaError_t launch_extrema(int precision, const void* prev, const void* phi, const Geom& gm, const CoefSet& cs,
                           double* out, cudaStream_t s);

// Bytes of one state buffer (9 flow + 5 thermal planes) and of a porosity field.
size_t state_buffer_bytes(int precision, int plane);
size_t phi_bytes(int precision, int plane);

// Adds the number of the n values of in outside (0, 1), NaN included, to *bad.
cudaError_t launch_count_bad_phi(const void* in, int in_is_double, long n, unsigned long long* bad, int nblocks,
                                 cudaStream_t s);
cudaError_t launch_convert_phi(const void* in, int in_is_double, void* out, int precision, const Geom& gm,
                               int nblocks, cudaStream_t s);

}  // namespace lbm
