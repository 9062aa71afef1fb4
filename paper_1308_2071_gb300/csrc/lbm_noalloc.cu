// lbm_observables_noalloc: the observables reduction of lbm_observables over
// a lattice state that the caller already holds in its own device memory,
// without any device allocation.  The reduction's scratch (the FP64 partial
// sums of every block, the result and a status word) lives in one file-scope
// static device array that every device loading the library keeps until the
// process exits.
#include <math.h>
#include <string.h>

#include <mutex>

#include "lbm_internal.h"

using namespace lbm;

namespace {

// 4 partial sums per block of the fixed reduction grid, 8 result slots, and
// one slot holding the (always clear) status word read by the finisher.
constexpr int kScratchDoubles = 4 * kReduceBlocks + 8 + 1;
constexpr size_t kScratchBytes = sizeof(double) * kScratchDoubles;
static_assert(kScratchBytes == 38984, "the header states the scratch size");

__device__ __align__(256) double g_obs_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_dev[kMaxDevices] = {nullptr};
int fail(int code, const std::string& msg) {
    set_global_error(msg);  // read back through lbm_last_error(NULL)
    return code;
}

// Device address of the static scratch on the current device.  In host code
// g_obs_scratch names a host-side stand-in, so the address is looked up once
// per device with that device current and cached.
int scratch_on_current_device(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LBM_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_obs_scratch);
        if (e != cudaSuccess || !p)
            return fail(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_dev[dev] = (double*)p;
    }
    *out = g_scratch_dev[dev];
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_observables_noalloc(const lbm_params* p, const void* ckpt_dev, size_t bytes, void* stream,
                            lbm_obs* out, void* ux_dev, void* uy_dev, void* T_dev, void* p_dev) {
    if (!p || !ckpt_dev || !out) return fail(LBM_ERR_ARG, "params, checkpoint and out are required");
    if (p->use_phi_field) return fail(LBM_ERR_ARG, "a porosity field is not part of a checkpoint");
    Derived dv;
    CoefSet cs;
    Geom gm;
    std::string why;
    int rc = setup_lattice(p, &dv, &cs, &gm, &why);
    if (rc != LBM_OK) return fail(rc, why);
    const size_t buf = state_buffer_bytes(p->precision, gm.plane);
    if (bytes < sizeof(CkptHeader) + buf) return fail(LBM_ERR_ARG, "checkpoint smaller than this lattice needs");

    double* scratch = nullptr;
    rc = scratch_on_current_device(&scratch);
    if (rc != LBM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;

    CkptHeader hd;
    cudaError_t e = cudaMemcpyAsync(&hd, ckpt_dev, sizeof hd, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("header read: ") + cudaGetErrorString(e));
    if (memcmp(hd.magic, "LBMCKPT", 8) != 0 || hd.version < 1 || hd.version > 3 ||
        !ckpt_layout_current(hd.version, hd.precision))
        return fail(LBM_ERR_ARG, "not a checkpoint of the current storage layout");
    // every version starts with B_{n-1}, the only buffer read here
    const long nbuf = hd.version == 1 ? 2 : 1;
    if (hd.nx != p->nx || hd.ny != p->ny || hd.precision != p->precision || hd.payload != (long)(nbuf * buf) ||
        bytes < sizeof(CkptHeader) + nbuf * buf)
        return fail(LBM_ERR_ARG, "checkpoint does not match the parameters");

    double* partials = scratch;
    double* result = scratch + 4 * kReduceBlocks;
    int* status = (int*)(scratch + 4 * kReduceBlocks + 8);
    // the array keeps the previous call's contents: clear the status word
    e = cudaMemsetAsync(status, 0, sizeof(double), s);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("status clear: ") + cudaGetErrorString(e));

    ObserveLaunch L;
    L.precision = p->precision;
    L.prev = (const char*)ckpt_dev + sizeof(CkptHeader);  // B_{n-1}: rebuilds the post-stream state S_n
    L.phi = nullptr;
    L.gm = gm;
    L.ux = ux_dev;
    L.uy = uy_dev;
    L.T = T_dev;
    L.p = p_dev;
    L.snap = nullptr;
    L.snap_valid = 0;
    L.partials = partials;
    L.nblocks = kReduceBlocks;
    L.L = dv.L;
    L.dT = dv.dT;
    L.status = status;
    L.out = result;
    L.stream = s;
    e = launch_observe(L, cs);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("observables: ") + cudaGetErrorString(e));
    double o[7];
    e = cudaMemcpyAsync(o, result, sizeof o, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("result read: ") + cudaGetErrorString(e));
    const double n = (double)p->nx * (double)p->ny;
    out->t = hd.t;
    out->nu_hot = o[0];
    out->nu_cold = o[1];
    out->umax = o[2];
    out->residual = 0.0;
    out->mass = n + o[4];
    out->heat = n * dv.T0 + o[5];
    // the state's own divergence test (the step kernels' flag is not part of a
    // checkpoint): a non-finite value or |u| >= 1/2 anywhere; a NaN anywhere
    // makes the maximum NaN
    const bool diverged = !(o[2] < 0.5) || !isfinite(o[4]) || !isfinite(o[5]);
    out->status = diverged ? LBM_ERR_DIVERGED : LBM_OK;
    if (diverged) return fail(LBM_ERR_DIVERGED, "the checkpoint holds a non-finite value or |u| >= 1/2");
    return LBM_OK;
}

}  // extern "C"
