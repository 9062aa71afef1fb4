// C-ABI runtime of liblbm (declared in include/lbm.h): parameter set-up of
// Section 4, state buffers, CUDA-graph replay of long step sequences and the
// observables round trip.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr int kGraphSteps = 64;  // steps per captured graph (even: keeps buffer parity)

thread_local std::string g_init_error;

}  // namespace

struct lbm_handle_s {
    lbm_params p;
    Derived dv;
    CoefSet coef;
    Geom gm;
    int precision;
    size_t buf_bytes;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;  // buf[cur] holds B_n, buf[cur ^ 1] holds B_{n-1}
    long t = 0;
    void* phi = nullptr;
    void* snap = nullptr;
    int snap_valid = 0;
    double* partials = nullptr;
    double* obs_dev = nullptr;
    double* obs_host = nullptr;
    int* status_dev = nullptr;
    unsigned* nu_counter = nullptr;  // block counter of the row-parallel Nusselt kernel
    double* nu_dev = nullptr;        // its two results
    double* wall_cols = nullptr;     // two halves of kObsCols temperatures per row, written by observing steps
    cudaStream_t nu_stream = nullptr;  // lbm_step_nusselt's reductions, beside the next step
    cudaEvent_t nu_step[2] = {nullptr, nullptr};  // observing step done, per half of wall_cols
    cudaEvent_t nu_red[2] = {nullptr, nullptr};   // its reduction done
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaGraphExec_t steady_exec = nullptr;
    long steady_key[4] = {0, 0, 0, 0};  // K, parity, max_checks, tol bits
    double* steady_dev = nullptr;       // 8 doubles of loop state
    double* extrema_dev = nullptr;      // 3 doubles per column
    int bx = 128, by = 2, npt = 1;
    std::string err;
};

namespace {

int fail(lbm_handle h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_init_error = msg;
    return code;
}

int cuda_fail(lbm_handle h, cudaError_t e, const char* where) {
    return fail(h, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(h, expr)                                          \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #expr); \
    } while (0)

// Section 4 set-up: Eq. 37 (second occurrence) for tau_nu and tau_T,
// Eq. 24 for nu_e, J = nu_e / nu, U = sqrt(g beta dT L) = Ma c_s, Da = K/L^2,
// Eq. 5 for F_phi.
int derive(const lbm_params* p, Derived* dv, std::string* why) {
    if (p->nx < 5 || p->ny < 5) return *why = "nx and ny must be >= 5", LBM_ERR_ARG;
    if (!(p->phi > 0.0 && p->phi <= 1.0)) return *why = "phi must lie in (0, 1]", LBM_ERR_ARG;
    const bool cooled = p->thermal_bc == LBM_BC_COOLED;
    if (!(p->Da > 0.0) || !(p->Pr > 0.0) || !(p->J > 0.0) || !(p->Ma > 0.0) || !(p->RaI >= 0.0))
        return *why = "Da, Pr, J and Ma must be positive and RaI non-negative", LBM_ERR_ARG;
    if (cooled ? !(p->RaI > 0.0) : !(p->Ra > 0.0))
        return *why = "Ra must be positive (RaI for LBM_BC_COOLED)", LBM_ERR_ARG;
    if (!(p->sigma > 0.0) || !(p->varpi < 1.0) || !(p->varpi > -4.0))
        return *why = "sigma must be positive and varpi in (-4, 1)", LBM_ERR_ARG;
    if (!(p->Th > p->Tc)) return *why = "Th must exceed Tc (with LBM_BC_COOLED, Th - Tc is the scale dT)", LBM_ERR_ARG;
    if (p->precision < LBM_F64 || p->precision > LBM_F32_FRAMED) return *why = "bad precision", LBM_ERR_ARG;
    if (p->use_phi_field && !(p->phi < 1.0))
        return *why = "a porosity field needs a mean porosity below 1", LBM_ERR_ARG;
    if (p->adiabatic_order != 1 && p->adiabatic_order != 2) return *why = "adiabatic_order is 1 or 2", LBM_ERR_ARG;
    if (p->thermal_bc != LBM_BC_SIDE_HEATED && p->thermal_bc != LBM_BC_COOLED)
        return *why = "unknown thermal_bc", LBM_ERR_ARG;
    if (p->collision != LBM_MRT && p->collision != LBM_LBGK) return *why = "unknown collision", LBM_ERR_ARG;
    const double cs2 = 1.0 / 3.0, cs = sqrt(cs2);
    const double L = (double)(p->nx - 1);
    const double cT2 = (4.0 + p->varpi) / 10.0;
    dv->L = L;
    // Eq. 37 (second occurrence); Section 4.2 replaces Ra by Ra_I when Ra = 0
    const double Rs = cooled ? p->RaI : p->Ra;
    dv->tau_nu = 0.5 + p->Ma * p->J * L / cs * sqrt(p->Pr / Rs);
    dv->tau_T = 0.5 + cs2 * (dv->tau_nu - 0.5) / (p->sigma * cT2 * p->Pr);
    if (!(dv->tau_nu > 0.5) || !(dv->tau_T > 0.5)) return *why = "relaxation time not above 1/2", LBM_ERR_ARG;
    dv->nu = cs2 * (dv->tau_nu - 0.5) / p->J;
    dv->dT = p->Th - p->Tc;
    const double U = p->Ma * cs;
    dv->gbeta = U * U / (dv->dT * L);
    dv->K = p->Da * L * L;
    dv->Fphi = p->forchheimer ? 1.75 / sqrt(150.0 * p->phi * p->phi * p->phi) : 0.0;
    // buoyancy reference: the mean wall temperature (Section 4.1), T_c with internal heating only (Section 4.2)
    dv->T0 = cooled ? p->Tc : 0.5 * (p->Th + p->Tc);
    // heat source: Ra_I / Ra = Q L^2 / (alpha_e dT) (Section 2), alpha_e from A9
    const double alpha = p->sigma * cT2 * (dv->tau_T - 0.5);
    if (cooled) dv->Q = dv->dT * alpha / (L * L);
    else if (p->RaI > 0.0) dv->Q = p->RaI / p->Ra * alpha * dv->dT / (L * L);
    else dv->Q = p->Qppp;
    return LBM_OK;
}

template <class R>
void fill_coef(const lbm_params* p, const Derived& dv, Coef<R>* c) {
    double s[9], z[5];
    if (p->collision == LBM_LBGK) {
        for (int k = 0; k < 9; ++k) s[k] = 1.0 / dv.tau_nu;
        for (int k = 0; k < 5; ++k) z[k] = 1.0 / dv.tau_T;
    } else {  // Section 4 choices
        const double sm[9] = {1.0, 1.1, 1.1, 1.0, 1.2, 1.0, 1.2, 1.0 / dv.tau_nu, 1.0 / dv.tau_nu};
        const double zm[5] = {1.0, 1.0 / dv.tau_T, 1.0 / dv.tau_T, 1.5, 1.5};
        memcpy(s, sm, sizeof s);
        memcpy(z, zm, sizeof z);
    }
    for (int k = 0; k < 9; ++k) {
        c->s[k] = (R)s[k];
        c->hs[k] = (R)(1.0 - 0.5 * s[k]);
    }
    for (int k = 0; k < 5; ++k) {
        c->z[k] = (R)z[k];
        c->hz[k] = (R)(1.0 - 0.5 * z[k]);
    }
    c->gbeta = (R)dv.gbeta;
    c->T0 = (R)dv.T0;
    c->dTh = (R)(p->Th - dv.T0);
    c->dTc = (R)(p->Tc - dv.T0);
    c->inv_sigma = (R)(1.0 / p->sigma);
    c->varpi = (R)p->varpi;
    c->inv_csT2 = (R)(10.0 / (4.0 + p->varpi));
    c->wt0 = (R)((1.0 - p->varpi) / 5.0);
    c->wt1 = (R)((4.0 + p->varpi) / 20.0);
    c->psi0 = (R)(dv.Q / p->sigma);
    c->psi3 = (R)(p->varpi * dv.Q / p->sigma);
    c->qhalf = (R)(0.5 * dv.Q / p->sigma);
    c->phi = (R)p->phi;
    c->c_lin = (R)(p->phi * dv.nu / dv.K);  // 0 when Da = INFINITY
    c->c_quad = (R)(p->phi * dv.Fphi / sqrt(dv.K));
    // per-cell Ergun (Eq. 5) with d_p^2 fixed by K(phi_bar) = K_bar:
    // phi nu / K(phi) = 150 nu (1-phi)^2 / (phi^2 d_p^2), phi F_phi / sqrt K = 1.75 (1-phi) / (phi^2 d_p)
    if (p->phi < 1.0) {
        const double pb = p->phi;
        const double dp2 = 150.0 * dv.K * (1.0 - pb) * (1.0 - pb) / (pb * pb * pb);
        c->a_lin = (R)(150.0 * dv.nu / dp2);
        c->a_quad = (R)(p->forchheimer ? 1.75 / sqrt(dp2) : 0.0);
    } else {
        c->a_lin = (R)0;
        c->a_quad = (R)0;
    }
    // 8-bit temperature frames: the power of two fq whose 128 steps span the
    // largest |T - T0| expected, the wall temperatures plus the conduction
    // maximum Q L^2 / (8 alpha_e) of a heat source (alpha_e from A9); a
    // larger |T - T0| only saturates the frame, which costs precision, not
    // correctness
    const double alpha = p->sigma * (4.0 + p->varpi) / 10.0 * (dv.tau_T - 0.5);
    const double tspan = fmax(fabs(p->Th - dv.T0), fabs(p->Tc - dv.T0)) + fabs(dv.Q) * dv.L * dv.L / (8.0 * alpha);
    const double fq = exp2(ceil(log2(tspan / 128.0)));
    c->fq = (R)fq;
    c->ifq = (R)(1.0 / fq);
    c->wt1fq = (R)((4.0 + p->varpi) / 20.0) * (R)fq;
}

}  // namespace

#ifdef LBM_BOUNDS_CHECK
// Bounds-checked build: the count of skipped out-of-plane accesses of every
// kernel of this process on this device (the symbol's device address is
// looked up on the host, so that nothing is allocated for it).
__device__ int g_oob_count;
#endif

namespace lbm {
void set_global_error(const std::string& msg) { g_init_error = msg; }

int* oob_counter() {
#ifdef LBM_BOUNDS_CHECK
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_oob_count) != cudaSuccess) return nullptr;
    return (int*)p;
#else
    return nullptr;
#endif
}

int setup_lattice(const lbm_params* p, Derived* dv, CoefSet* cs, Geom* gm, std::string* why) {
    int rc = derive(p, dv, why);
    if (rc != LBM_OK) return rc;
    // row pitch in elements: rows of the flow planes and of the thermal planes
    // both start on 128-byte boundaries (FP64: 16, FP32: 32, FP16 flow: 64)
    const int align = p->precision == LBM_F64 ? 16 : (p->precision == LBM_F32_STORE_F16 ? 64 : 32);
    const long pitch = ((long)p->nx + align - 1) / align * align;
    const long plane = pitch * (long)p->ny;
    if (plane * NPOP >= (1L << 31)) return *why = "lattice too large for 32-bit offsets", LBM_ERR_ARG;
    gm->nx = p->nx;
    gm->ny = p->ny;
    gm->pitch = (int)pitch;
    gm->plane = (int)plane;
    gm->thermal_bc = p->thermal_bc;
    gm->adi_order = p->adiabatic_order;
#ifdef LBM_BOUNDS_CHECK
    gm->oob = oob_counter();
    if (!gm->oob) return *why = "bounds-checked build: no device counter", LBM_ERR_CUDA;
#endif
    fill_coef<double>(p, *dv, &cs->d);
    fill_coef<float>(p, *dv, &cs->f);
    return LBM_OK;
}
}  // namespace lbm

namespace {

void free_handle(lbm_handle h) {
    if (!h) return;
    for (int k = 0; k < 2; ++k) {
        if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
        if (h->buf[k]) cudaFree(h->buf[k]);
    }
    if (h->steady_exec) cudaGraphExecDestroy(h->steady_exec);
    if (h->steady_dev) cudaFree(h->steady_dev);
    if (h->extrema_dev) cudaFree(h->extrema_dev);
    if (h->phi) cudaFree(h->phi);
    if (h->snap) cudaFree(h->snap);
    if (h->partials) cudaFree(h->partials);
    if (h->obs_dev) cudaFree(h->obs_dev);
    if (h->status_dev) cudaFree(h->status_dev);
    if (h->nu_counter) cudaFree(h->nu_counter);
    if (h->nu_dev) cudaFree(h->nu_dev);
    if (h->wall_cols) cudaFree(h->wall_cols);
    for (int b = 0; b < 2; ++b) {
        if (h->nu_step[b]) cudaEventDestroy(h->nu_step[b]);
        if (h->nu_red[b]) cudaEventDestroy(h->nu_red[b]);
    }
    if (h->nu_stream) cudaStreamDestroy(h->nu_stream);
    if (h->obs_host) cudaFreeHost(h->obs_host);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

StepLaunch step_launch(lbm_handle h, int src, cudaStream_t s) {
    StepLaunch L;
    L.precision = h->precision;
    L.src = h->buf[src];
    L.dst = h->buf[src ^ 1];
    L.phi = h->p.use_phi_field ? h->phi : nullptr;
    L.gm = h->gm;
    L.bx = h->bx;
    L.by = h->by;
    L.npt = h->npt;
    L.status = h->status_dev;
    L.stream = s;
    return L;
}

// nsteps steps from buf[cur] in the handle's launch shape, the first launched
// as a programmatic dependent when pdl_first (a step kernel right before it).
int advance(lbm_handle h, long nsteps, bool pdl_first) {
    for (long k = 0; k < nsteps; ++k) {
        StepLaunch Ls = step_launch(h, h->cur, h->stream);
        Ls.pdl = k > 0 || pdl_first;
        CK(h, launch_step(Ls, h->coef));
        h->cur ^= 1;
    }
    return LBM_OK;
}

// State B_{-1} = rest everywhere (zero deviations) in both buffers, then one
// step: pulling the rest state and applying the wall rule gives the initial
// post-stream state S_0, whose collision is B_0.
int reset_state(lbm_handle h) {
    CK(h, cudaMemsetAsync(h->buf[0], 0, h->buf_bytes, h->stream));
    CK(h, cudaMemsetAsync(h->buf[1], 0, h->buf_bytes, h->stream));
    CK(h, cudaMemsetAsync(h->status_dev, 0, sizeof(int), h->stream));
    h->cur = 0;
    CK(h, launch_step(step_launch(h, 0, h->stream), h->coef));
    h->cur = 1;
    h->t = 0;
    h->snap_valid = 0;
    return LBM_OK;
}

int capture_graph(lbm_handle h, int parity) {
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int src = parity;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) {
        e = launch_step(step_launch(h, src, h->cap_stream), h->coef);
        src ^= 1;
    }
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h, e, "capture step");
    }
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->gexec[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    return LBM_OK;
}

void drop_graphs(lbm_handle h) {
    for (int k = 0; k < 2; ++k)
        if (h->gexec[k]) {
            cudaGraphExecDestroy(h->gexec[k]);
            h->gexec[k] = nullptr;
        }
    if (h->steady_exec) {
        cudaGraphExecDestroy(h->steady_exec);
        h->steady_exec = nullptr;
    }
}

// The steady-state graph: while (cond) { K steps; check }.
int build_steady_graph(lbm_handle h, long K, long max_checks, double tol) {
    cudaGraph_t g = nullptr;
    CK(h, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            int src = h->cur;
            for (long k = 0; k < K && e == cudaSuccess; ++k) {
                e = launch_step(step_launch(h, src, h->cap_stream), h->coef);
                src ^= 1;
            }
            if (e == cudaSuccess) {
                SteadyCheckLaunch L;
                L.precision = h->precision;
                L.prev = h->buf[h->cur ^ 1];
                L.gm = h->gm;
                L.L = h->dv.L;
                L.dT = h->dv.dT;
                L.status = h->status_dev;
                L.tol = tol;
                L.max_checks = max_checks;
                L.state = h->steady_dev;
                L.cond = cond;
                L.stream = h->cap_stream;
                e = launch_steady_check(L, h->coef);
            }
            cudaGraph_t out = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &out);
            if (e == cudaSuccess) e = e2;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->steady_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "steady-state graph");
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_params_default(lbm_params* p, int nx, int ny, double Ra, double Da, double phi) {
    memset(p, 0, sizeof(*p));
    p->nx = nx;
    p->ny = ny;
    p->Ra = Ra;
    p->Da = Da;
    p->phi = phi;
    p->Pr = 1.0;
    p->J = 1.0;
    p->Ma = 0.1;
    p->sigma = 1.0;
    p->varpi = -2.0;
    p->Th = 1.0;
    p->Tc = 0.0;
    p->Qppp = 0.0;
    p->precision = LBM_F32;
    p->use_phi_field = 0;
    p->forchheimer = 1;
    p->thermal_bc = LBM_BC_SIDE_HEATED;
    p->adiabatic_order = 1;
    p->collision = LBM_MRT;
    p->block_x = 0;
    p->block_y = 0;
}

int lbm_init(const lbm_params* p, void* stream, lbm_handle* out) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, LBM_ERR_ARG, "params is NULL");
    lbm_handle h = new lbm_handle_s();
    std::string why;
    int rc = setup_lattice(p, &h->dv, &h->coef, &h->gm, &why);
    if (rc != LBM_OK) {
        delete h;
        return fail(nullptr, rc, why);
    }
    h->p = *p;
    h->precision = p->precision;
    const long plane = h->gm.plane;
    // defaults (the autotuner's picks on the 4096^2 benchmark lattice): FP32
    // arithmetic two nodes side by side along x in 128-thread blocks, FP64 two
    // nodes along y
    h->bx = p->block_x > 0 ? p->block_x : (p->nx <= 128 ? 32 : 64);
    h->by = p->block_y > 0 ? p->block_y : (h->bx >= 128 ? 1 : 128 / h->bx);
    h->npt = p->nodes_per_thread > 0 ? p->nodes_per_thread : (p->precision == LBM_F64 ? 2 : 3);
    if (h->bx * h->by > 256 || h->bx <= 0 || h->by <= 0 || h->npt > 3) {
        delete h;
        return fail(nullptr, LBM_ERR_ARG, "block_x * block_y must be <= 256 and nodes_per_thread 1, 2 or 3");
    }
    h->stream = (cudaStream_t)stream;
    h->buf_bytes = state_buffer_bytes(p->precision, (int)plane);

    cudaError_t e;
#define CKI(expr)                                                   \
    do {                                                            \
        e = (expr);                                                 \
        if (e != cudaSuccess) {                                     \
            std::string m_ = std::string(#expr) + ": " + cudaGetErrorString(e); \
            free_handle(h);                                         \
            return fail(nullptr, LBM_ERR_CUDA, m_);                 \
        }                                                           \
    } while (0)
    CKI(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CKI(cudaMalloc(&h->buf[0], h->buf_bytes));
    CKI(cudaMalloc(&h->buf[1], h->buf_bytes));
    CKI(cudaMalloc(&h->partials, sizeof(double) * 4 * kReduceBlocks));
    CKI(cudaMalloc(&h->obs_dev, sizeof(double) * 8));
    CKI(cudaMalloc(&h->status_dev, sizeof(int)));
    CKI(cudaMalloc(&h->nu_counter, sizeof(unsigned)));
    CKI(cudaMemsetAsync(h->nu_counter, 0, sizeof(unsigned), h->stream));
    CKI(cudaMalloc(&h->nu_dev, 2 * sizeof(double)));
    CKI(cudaMalloc(&h->wall_cols, sizeof(double) * 2 * kObsCols * (size_t)p->ny));
    CKI(cudaMallocHost(&h->obs_host, sizeof(double) * 8));
    const size_t rsz = p->precision == LBM_F64 ? 8 : 4;
    CKI(cudaMalloc(&h->snap, rsz * 2 * (size_t)p->nx * p->ny));
    if (p->use_phi_field) {
        CKI(cudaMalloc(&h->phi, phi_bytes(p->precision, (int)plane)));
        CKI(cudaMemsetAsync(h->phi, 0, phi_bytes(p->precision, (int)plane), h->stream));
    }
#undef CKI
    if (p->use_phi_field) {
        // until a field is set, every cell holds the mean porosity
        std::string m;
        const size_t n = (size_t)p->nx * p->ny;
        double* tmp = nullptr;
        e = cudaMalloc(&tmp, n * sizeof(double));
        if (e == cudaSuccess) {
            double* host = (double*)malloc(n * sizeof(double));
            for (size_t k = 0; k < n; ++k) host[k] = p->phi;
            e = cudaMemcpyAsync(tmp, host, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess)
                e = launch_convert_phi(tmp, 1, h->phi, h->precision, h->gm, kReduceBlocks, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            free(host);
            cudaFree(tmp);
        }
        if (e != cudaSuccess) {
            m = std::string("porosity fill: ") + cudaGetErrorString(e);
            free_handle(h);
            return fail(nullptr, LBM_ERR_CUDA, m);
        }
    }
    rc = reset_state(h);
    if (rc != LBM_OK) {
        std::string m = h->err;
        free_handle(h);
        return fail(nullptr, rc, m);
    }
    *out = h;
    return LBM_OK;
}

int lbm_set_porous_field(lbm_handle h, const void* phi_dev, int dtype) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!h->p.use_phi_field) return fail(h, LBM_ERR_STATE, "handle was created with use_phi_field = 0");
    if (!phi_dev) return fail(h, LBM_ERR_ARG, "phi_dev is NULL");
    if (dtype != LBM_F64 && dtype != LBM_F32) return fail(h, LBM_ERR_ARG, "dtype must be LBM_F64 or LBM_F32");
    // every cell must lie in (0, 1): a 0 would make 1/phi infinite, a 1 or more
    // the Ergun drag zero or negative (Eq. 5); the count lands in the
    // partial-sum scratch, which no other call uses concurrently
    unsigned long long* bad = (unsigned long long*)h->partials;
    unsigned long long nbad = 0;
    CK(h, cudaMemsetAsync(bad, 0, sizeof *bad, h->stream));
    CK(h, launch_count_bad_phi(phi_dev, dtype == LBM_F64, (long)h->p.nx * h->p.ny, bad, kReduceBlocks, h->stream));
    CK(h, cudaMemcpyAsync(h->obs_host, bad, sizeof nbad, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    memcpy(&nbad, h->obs_host, sizeof nbad);
    if (nbad) return fail(h, LBM_ERR_ARG, std::to_string(nbad) + " porosity values outside (0, 1)");
    CK(h, launch_convert_phi(phi_dev, dtype == LBM_F64, h->phi, h->precision, h->gm, kReduceBlocks, h->stream));
    drop_graphs(h);
    return reset_state(h);
}

int lbm_bounds_check(int* enabled, long* count) {
#ifdef LBM_BOUNDS_CHECK
    if (enabled) *enabled = 1;
    int* p = oob_counter();
    if (!p) return fail(nullptr, LBM_ERR_CUDA, "bounds-checked build: no device counter");
    int v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p, 0, sizeof v);
    if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, std::string("bounds counter: ") + cudaGetErrorString(e));
    if (count) *count = v;
#else
    if (enabled) *enabled = 0;
    if (count) *count = 0;
#endif
    return LBM_OK;
}

int lbm_reset(lbm_handle h) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    return reset_state(h);
}

int lbm_tune(lbm_handle h, const char* cache_path, int* block_x, int* block_y, int* nodes_per_thread) {
    TraceRange trace_("lbm_tune");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    char sig[256];
    {
        int dev = 0;
        cudaDeviceProp pr;
        std::string name = "unknown";
        if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&pr, dev) == cudaSuccess) name = pr.name;
        for (auto& ch : name)
            if (ch == ' ') ch = '_';
        snprintf(sig, sizeof sig, "step:%s:p%d:%dx%d:f%d", name.c_str(), h->precision, h->p.nx, h->p.ny,
                 h->p.use_phi_field);
    }
    int best[3] = {h->bx, h->by, h->npt};
    bool cached = false;
    if (cache_path) {
        FILE* fp = fopen(cache_path, "r");
        if (fp) {
            char key[256];
            int a, b, c;
            while (fscanf(fp, "%255s %d %d %d", key, &a, &b, &c) == 4)
                if (strcmp(key, sig) == 0) {
                    best[0] = a;
                    best[1] = b;
                    best[2] = c;
                    cached = true;
                }
            fclose(fp);
        }
    }
    if (!cached) {
        const int cand[][3] = {{128, 2, 1}, {64, 4, 1}, {256, 1, 1}, {32, 8, 1}, {128, 1, 2}, {64, 2, 2},
                               {128, 2, 2}, {256, 1, 2}, {32, 4, 2}, {32, 8, 3}, {64, 4, 3}, {128, 2, 3},
                               {64, 2, 3},  {128, 1, 3}, {256, 1, 3}};
        cudaEvent_t e0, e1;
        CK(h, cudaEventCreate(&e0));
        CK(h, cudaEventCreate(&e1));
        float best_ms = 1e30f;
        drop_graphs(h);
        for (auto& cd : cand) {
            h->bx = cd[0];
            h->by = cd[1];
            h->npt = cd[2];
            int rc = advance(h, 3, false);
            if (rc != LBM_OK) return rc;
            // 30 steps, or on small lattices as many as take about 2 ms (at most
            // 2000), so that timer resolution and clock ramps do not pick the shape
            long nsteps = 30;
            float ms = 0.f;
            for (int pass = 0; pass < 2; ++pass) {
                CK(h, cudaEventRecord(e0, h->stream));
                if ((rc = advance(h, nsteps, false)) != LBM_OK) return rc;
                CK(h, cudaEventRecord(e1, h->stream));
                CK(h, cudaEventSynchronize(e1));
                CK(h, cudaEventElapsedTime(&ms, e0, e1));
                if (pass == 1 || ms >= 2.f) break;
                nsteps = std::min(2000L, (long)(nsteps * 2.f / std::max(ms, 1e-3f)) + 1);
            }
            ms *= 30.f / (float)nsteps;  // per 30 steps
            if (ms < best_ms) {
                best_ms = ms;
                best[0] = cd[0];
                best[1] = cd[1];
                best[2] = cd[2];
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (cache_path) {
            FILE* fp = fopen(cache_path, "a");
            if (fp) {
                fprintf(fp, "%s %d %d %d\n", sig, best[0], best[1], best[2]);
                fclose(fp);
            }
        }
    }
    h->bx = best[0];
    h->by = best[1];
    h->npt = best[2];
    drop_graphs(h);
    int rc = reset_state(h);
    if (rc != LBM_OK) return rc;
    if (block_x) *block_x = best[0];
    if (block_y) *block_y = best[1];
    if (nodes_per_thread) *nodes_per_thread = best[2];
    return LBM_OK;
}

int lbm_step(lbm_handle h, long nsteps) {
    TraceRange trace_("lbm_step");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (nsteps < 0) return fail(h, LBM_ERR_ARG, "nsteps < 0");
    long left = nsteps;
    while (left >= kGraphSteps) {
        if (!h->gexec[h->cur]) {
            int rc = capture_graph(h, h->cur);
            if (rc != LBM_OK) return rc;
        }
        CK(h, cudaGraphLaunch(h->gexec[h->cur], h->stream));
        left -= kGraphSteps;  // even count: cur unchanged
    }
    for (long k = 0; left > 0; --left, ++k) {
        StepLaunch Ls = step_launch(h, h->cur, h->stream);
        Ls.pdl = k > 0;  // directly behind the previous step kernel
        CK(h, launch_step(Ls, h->coef));
        h->cur ^= 1;
    }
    h->t += nsteps;
    return LBM_OK;
}

int lbm_observables(lbm_handle h, lbm_obs* out, void* ux_dev, void* uy_dev, void* T_dev, void* p_dev) {
    TraceRange trace_("lbm_observables");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    ObserveLaunch L;
    L.precision = h->precision;
    L.prev = h->buf[h->cur ^ 1];
    L.phi = h->p.use_phi_field ? h->phi : nullptr;
    L.gm = h->gm;
    L.ux = ux_dev;
    L.uy = uy_dev;
    L.T = T_dev;
    L.p = p_dev;
    L.snap = h->snap;
    L.snap_valid = h->snap_valid;
    L.partials = h->partials;
    L.nblocks = kReduceBlocks;
    L.L = h->dv.L;
    L.dT = h->dv.dT;
    L.status = h->status_dev;
    L.out = h->obs_dev;
    L.stream = h->stream;
    CK(h, launch_observe(L, h->coef));
    CK(h, cudaMemcpyAsync(h->obs_host, h->obs_dev, sizeof(double) * 7, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->snap_valid = 1;
    const double* o = h->obs_host;
    const double n = (double)h->p.nx * (double)h->p.ny;
    const int status = o[6] != 0.0 ? LBM_ERR_DIVERGED : LBM_OK;
    if (out) {
        out->t = h->t;
        out->nu_hot = o[0];
        out->nu_cold = o[1];
        out->umax = o[2];
        out->residual = o[2] > 0.0 ? o[3] / o[2] : 0.0;
        out->mass = n + o[4];  // sum_i w_i rho0 = 1 per node
        out->heat = n * h->dv.T0 + o[5];
        out->status = status;
    }
    if (status != LBM_OK) return fail(h, status, "divergence flag raised (non-finite value or |u| >= 1/2)");
    return LBM_OK;
}

namespace {
// The address a kernel writes to for p: p itself for device and managed
// memory, the mapped device address for page-locked host memory, nullptr for
// pageable host memory or a pointer not aligned for doubles.
double* device_writable(double* p) {
    if ((uintptr_t)p % alignof(double) != 0) return nullptr;
    cudaPointerAttributes a;
    memset(&a, 0, sizeof a);
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return (double*)a.devicePointer;
    return nullptr;
}

// out: where the kernel writes (nu_hot, nu_cold); device-accessible memory
int enqueue_nusselt(lbm_handle h, double* out) {
    if (4 * kReduceBlocks < 2 * ((h->p.ny + 31) / 32)) return fail(h, LBM_ERR_ARG, "too many rows for the reduction");
    ObserveLaunch L;
    memset(&L, 0, sizeof(L));
    L.precision = h->precision;
    L.prev = h->buf[h->cur ^ 1];
    L.gm = h->gm;
    L.partials = h->partials;
    L.L = h->dv.L;
    L.dT = h->dv.dT;
    L.status = h->status_dev;
    L.out = out;
    L.counter = h->nu_counter;
    L.stream = h->stream;
    CK(h, launch_nusselt(L, h->coef));
    return LBM_OK;
}
}  // namespace

int lbm_nusselt(lbm_handle h, double* nu_hot, double* nu_cold) {
    TraceRange trace_("lbm_nusselt");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    int rc = enqueue_nusselt(h, h->nu_dev);
    if (rc != LBM_OK) return rc;
    CK(h, cudaMemcpyAsync(h->obs_host, h->nu_dev, sizeof(double) * 2, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (nu_hot) *nu_hot = h->obs_host[0];
    if (nu_cold) *nu_cold = h->obs_host[1];
    return LBM_OK;
}

int lbm_nusselt_async(lbm_handle h, double* out2) {
    TraceRange trace_("lbm_nusselt_async");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!out2) return fail(h, LBM_ERR_ARG, "out2 is NULL");
    // device memory and mapped (pinned) host memory: the kernel writes there
    // itself; other host memory gets a copy
    double* direct = device_writable(out2);
    int rc = enqueue_nusselt(h, direct ? direct : h->nu_dev);
    if (rc != LBM_OK) return rc;
    if (!direct) CK(h, cudaMemcpyAsync(out2, h->nu_dev, sizeof(double) * 2, cudaMemcpyDefault, h->stream));
    return LBM_OK;
}

int lbm_step_nusselt(lbm_handle h, long nsteps, double* out) {
    TraceRange trace_("lbm_step_nusselt");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (nsteps < 0) return fail(h, LBM_ERR_ARG, "nsteps < 0");
    if (nsteps == 0) return LBM_OK;
    if (!out) return fail(h, LBM_ERR_ARG, "out is NULL");
    if (4 * kReduceBlocks < 2 * ((h->p.ny + 31) / 32)) return fail(h, LBM_ERR_ARG, "too many rows for the reduction");
    double* dev = device_writable(out);
    if (!dev) return fail(h, LBM_ERR_ARG, "out must be device memory or page-locked host memory, aligned for double");
    if (!h->nu_stream) {
        // the reductions take few blocks: the highest priority lets them in
        // while the next step's blocks are still being dispatched
        int least = 0, greatest = 0;
        CK(h, cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CK(h, cudaStreamCreateWithPriority(&h->nu_stream, cudaStreamNonBlocking, greatest));
        for (int b = 0; b < 2; ++b) {
            CK(h, cudaEventCreateWithFlags(&h->nu_step[b], cudaEventDisableTiming));
            CK(h, cudaEventCreateWithFlags(&h->nu_red[b], cudaEventDisableTiming));
        }
    }
    ObserveLaunch L;
    memset(&L, 0, sizeof(L));
    L.precision = h->precision;
    L.gm = h->gm;
    L.partials = h->partials;
    L.L = h->dv.L;
    L.dT = h->dv.dT;
    L.status = h->status_dev;
    L.counter = h->nu_counter;
    L.stream = h->nu_stream;
    // step k writes half k & 1 of wall_cols; its reduction runs on nu_stream
    // beside step k + 1 (which writes the other half), and step k + 2 waits
    // for it before rewriting the half
    cudaError_t e = cudaSuccess;
    const char* where = "";
    for (long k = 0; k < nsteps; ++k) {
        const int b = (int)(k & 1);
        double* cols = h->wall_cols + (size_t)b * kObsCols * h->p.ny;
        if (k >= 2 && (e = cudaStreamWaitEvent(h->stream, h->nu_red[b], 0)) != cudaSuccess) {
            where = "wait for the reduction two steps back";
            break;
        }
        StepLaunch Ls = step_launch(h, h->cur, h->stream);
        Ls.obs = cols;
        if ((e = launch_step(Ls, h->coef)) != cudaSuccess) {
            where = "observing step";
            break;
        }
        h->cur ^= 1;
        h->t += 1;
        if ((e = cudaEventRecord(h->nu_step[b], h->stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(h->nu_stream, h->nu_step[b], 0)) != cudaSuccess) {
            where = "hand-over to the reduction stream";
            break;
        }
        L.prev = h->buf[h->cur ^ 1];
        L.obs = cols;
        L.out = dev + 2 * k;
        if ((e = launch_nusselt(L, h->coef)) != cudaSuccess ||
            (e = cudaEventRecord(h->nu_red[b], h->nu_stream)) != cudaSuccess) {
            where = "wall-column reduction";
            break;
        }
    }
    // the caller's stream reaches this point once the last reduction is done
    // (the reductions run in order on nu_stream)
    if (e == cudaSuccess && (e = cudaStreamWaitEvent(h->stream, h->nu_red[(nsteps - 1) & 1], 0)) != cudaSuccess)
        where = "join of the reduction stream";
    if (e != cudaSuccess) {
        (void)cudaStreamSynchronize(h->nu_stream);  // no reduction keeps running beside later work
        return cuda_fail(h, e, where);
    }
    return LBM_OK;
}

int lbm_adjoint_step(lbm_handle h, long nsteps, long ckpt_every, double* J, void* dJdphi_dev) {
    TraceRange trace_("lbm_adjoint_step");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!h->p.use_phi_field) return fail(h, LBM_ERR_STATE, "the adjoint needs a handle created with use_phi_field = 1");
    if (h->precision != LBM_F64 && h->precision != LBM_F32 && h->precision != LBM_F32_FRAMED)
        return fail(h, LBM_ERR_ARG, "the adjoint runs in LBM_F64, LBM_F32 or LBM_F32_FRAMED");
    if (h->p.adiabatic_order != 1) return fail(h, LBM_ERR_ARG, "the adjoint supports first-order adiabatic walls");
    if (nsteps < 1 || ckpt_every < 1 || !dJdphi_dev) return fail(h, LBM_ERR_ARG, "need nsteps >= 1, ckpt_every >= 1, output");
    const long N = nsteps, K = ckpt_every < nsteps ? ckpt_every : nsteps;
    const long nseg = (N + K - 1) / K;
    const size_t rsz = h->precision == LBM_F64 ? sizeof(double) : sizeof(float);
    void *ckpt = nullptr, *seg = nullptr, *madj = nullptr;
    double* gphi = nullptr;
    auto release = [&]() {
        if (ckpt) cudaFree(ckpt);
        if (seg) cudaFree(seg);
        if (madj) cudaFree(madj);
        if (gphi) cudaFree(gphi);
    };
    cudaError_t e = cudaMalloc(&ckpt, (size_t)nseg * h->buf_bytes);
    // two halves of K - 1 recomputed states: one segment is recomputed while the next is reversed
    if (e == cudaSuccess && K > 1) e = cudaMalloc(&seg, 2 * (size_t)(K - 1) * h->buf_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&madj, 2 * (size_t)h->gm.plane * NPOP * rsz);
    if (e == cudaSuccess) e = cudaMalloc(&gphi, sizeof(double) * (size_t)h->p.nx * h->p.ny);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(h, e, "adjoint buffers");
    }
    // forward sweep from the initial state, keeping B_{sK-1} (state index j = sK)
    int rc = reset_state(h);
    if (rc == LBM_OK) {
        e = cudaMemsetAsync(ckpt, 0, h->buf_bytes, h->stream);  // j = 0: the rest state B_{-1}
        if (e != cudaSuccess) rc = cuda_fail(h, e, "adjoint forward sweep");
        // runs of steps between the kept states: before step t (buf[cur] holds
        // B_t, state index j = t + 1) the state is kept when j % K == 0, j < N
        for (long t = 0; t < N && rc == LBM_OK;) {
            const long j = t + 1;
            const bool copy = j % K == 0 && j <= N - 1;
            if (copy && (e = cudaMemcpyAsync((char*)ckpt + (size_t)(j / K) * h->buf_bytes, h->buf[h->cur],
                                             h->buf_bytes, cudaMemcpyDeviceToDevice, h->stream)) != cudaSuccess) {
                rc = cuda_fail(h, e, "adjoint forward sweep");
                break;
            }
            const long next = (j / K + 1) * K - 1;  // the next step that keeps its input state
            const long upto = next <= N - 2 ? next : N;
            rc = advance(h, upto - t, t > 0 && !copy);  // directly behind the previous step kernel
            t = upto;
        }
        h->t = N;
    }
    if (rc == LBM_OK) {
        double nuh = 0.0;
        rc = lbm_nusselt(h, &nuh, nullptr);
        if (rc == LBM_OK && J) *J = nuh;
    }
    if (rc == LBM_OK) {
        AdjointJob A;
        A.precision = h->precision;
        A.gm = h->gm;
        A.coef = h->precision == LBM_F64 ? (const void*)&h->coef.d : (const void*)&h->coef.f;
        A.nsteps = N;
        A.ckpt_every = K;
        A.buf_bytes = h->buf_bytes;
        A.ckpt = ckpt;
        A.seg = seg;
        A.madj = madj;
        A.gphi = gphi;
        A.phi = h->phi;
        A.status = h->status_dev;
        A.L = h->dv.L;
        A.dT = h->dv.dT;
        A.out = dJdphi_dev;
        A.bx = h->bx;  // the handle's (tuned) launch shape, as in the forward sweep
        A.by = h->by;
        A.npt = h->npt;
        A.stream = h->stream;
        e = launch_adjoint_sweep(A);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "adjoint reverse sweep");
    }
    release();
    return rc;
}

int lbm_run_steady(lbm_handle h, double tol, long check_every, long max_steps, long* steps_taken, double* change) {
    TraceRange trace_("lbm_run_steady");
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!(tol > 0.0) || check_every < 1 || max_steps < 1) return fail(h, LBM_ERR_ARG, "need tol > 0, check_every >= 1, max_steps >= 1");
    const long K = (check_every + 1) / 2 * 2;  // even: the captured buffers return to their parity
    const long max_checks = (max_steps + K - 1) / K;
    if (!h->steady_dev) CK(h, cudaMalloc(&h->steady_dev, 8 * sizeof(double)));
    long tolbits;
    memcpy(&tolbits, &tol, sizeof tolbits);
    const long key[4] = {K, h->cur, max_checks, tolbits};
    if (!h->steady_exec || memcmp(key, h->steady_key, sizeof key) != 0) {
        if (h->steady_exec) cudaGraphExecDestroy(h->steady_exec);
        h->steady_exec = nullptr;
        int rc = build_steady_graph(h, K, max_checks, tol);
        if (rc != LBM_OK) return rc;
        memcpy(h->steady_key, key, sizeof key);
    }
    CK(h, cudaMemsetAsync(h->steady_dev, 0, 8 * sizeof(double), h->stream));
    CK(h, cudaGraphLaunch(h->steady_exec, h->stream));
    double st[8];
    CK(h, cudaMemcpyAsync(st, h->steady_dev, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const long steps = (long)st[3] * K;
    h->t += steps;
    h->snap_valid = 0;
    if (steps_taken) *steps_taken = steps;
    if (change) *change = st[2];
    if ((int)st[4] == 2) return fail(h, LBM_ERR_DIVERGED, "divergence flag raised during the steady-state loop");
    return LBM_OK;
}

int lbm_field_extrema(lbm_handle h, double* T_max, double* psi_min, double* psi_max) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!h->extrema_dev) CK(h, cudaMalloc(&h->extrema_dev, 3 * sizeof(double) * (size_t)h->p.nx));
    CK(h, launch_extrema(h->precision, h->buf[h->cur ^ 1], h->p.use_phi_field ? h->phi : nullptr, h->gm, h->coef,
                         h->extrema_dev, h->stream));
    std::vector<double> col(3 * (size_t)h->p.nx);
    CK(h, cudaMemcpyAsync(col.data(), h->extrema_dev, sizeof(double) * col.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    double tm = -INFINITY, pmn = 0.0, pmx = 0.0;
    for (int x = 0; x < h->p.nx; ++x) {
        tm = fmax(tm, col[3 * x]);
        pmn = fmin(pmn, col[3 * x + 1]);
        pmx = fmax(pmx, col[3 * x + 2]);
    }
    if (T_max) *T_max = tm;
    if (psi_min) *psi_min = pmn;
    if (psi_max) *psi_max = pmx;
    return LBM_OK;
}

int lbm_read_state(lbm_handle h, double* f_dev, double* g_dev) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!f_dev || !g_dev) return fail(h, LBM_ERR_ARG, "f_dev and g_dev are required");
    ReadStateLaunch L;
    L.precision = h->precision;
    L.prev = h->buf[h->cur ^ 1];
    L.phi = h->p.use_phi_field ? h->phi : nullptr;
    L.gm = h->gm;
    L.f = f_dev;
    L.g = g_dev;
    L.nblocks = kReduceBlocks;
    L.stream = h->stream;
    CK(h, launch_read_state(L, h->coef));
    return LBM_OK;
}

int lbm_checkpoint_size(lbm_handle h, size_t* bytes) {
    if (!h || !bytes) return fail(h, LBM_ERR_ARG, "handle and bytes are required");
    *bytes = sizeof(CkptHeader) + h->buf_bytes;
    return LBM_OK;
}

// Host-to-device copy of a checkpoint's payload.  From pinned memory the copy
// runs about 8 % faster from a 256-byte-aligned host address (211 against
// 194 GB/s measured on GB300 at the 40-byte header's offset), so the bytes
// before the next boundary go first, apart.
static cudaError_t copy_in(void* dst, const char* src, size_t n, cudaStream_t s) {
    size_t head = (256 - ((uintptr_t)src & 255)) & 255;
    if (head > n) head = n;
    if (head) {
        cudaError_t e = cudaMemcpyAsync(dst, src, head, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaMemcpyAsync((char*)dst + head, src + head, n - head, cudaMemcpyHostToDevice, s);
}

int lbm_save(lbm_handle h, void* host, size_t bytes) {
    TraceRange trace_("lbm_save");
    if (!h || !host) return fail(h, LBM_ERR_ARG, "handle and host buffer are required");
    size_t need = sizeof(CkptHeader) + h->buf_bytes;
    if (bytes < need) return fail(h, LBM_ERR_ARG, "checkpoint buffer too small");
    CkptHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, "LBMCKPT", 8);
    hd.version = 3;
    hd.nx = h->p.nx;
    hd.ny = h->p.ny;
    hd.precision = h->precision;
    hd.t = h->t;
    hd.payload = (long)h->buf_bytes;
    memcpy(host, &hd, sizeof hd);
    // B_{n-1} alone: the post-stream state S_n is pulled from it, and B_n is collide(S_n)
    CK(h, cudaMemcpyAsync((char*)host + sizeof hd, h->buf[h->cur ^ 1], h->buf_bytes, cudaMemcpyDeviceToHost,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_load(lbm_handle h, const void* host, size_t bytes) {
    TraceRange trace_("lbm_load");
    if (!h || !host) return fail(h, LBM_ERR_ARG, "handle and host buffer are required");
    CkptHeader hd;
    if (bytes < sizeof hd) return fail(h, LBM_ERR_ARG, "checkpoint buffer too small");
    memcpy(&hd, host, sizeof hd);
    if (memcmp(hd.magic, "LBMCKPT", 8) != 0 || hd.version < 1 || hd.version > 3)
        return fail(h, LBM_ERR_ARG, "not a checkpoint");
    if (!ckpt_layout_current(hd.version, hd.precision))
        return fail(h, LBM_ERR_ARG, "checkpoint written with an older storage layout of this precision");
    const long nbuf = hd.version == 1 ? 2 : 1;
    if (hd.nx != h->p.nx || hd.ny != h->p.ny || hd.precision != h->precision ||
        hd.payload != (long)(nbuf * h->buf_bytes) || bytes < sizeof hd + nbuf * h->buf_bytes)
        return fail(h, LBM_ERR_ARG, "checkpoint does not match this handle");
    const char* src = (const char*)host + sizeof hd;
    for (long k = 0; k < nbuf; ++k) CK(h, copy_in(h->buf[k], src + k * h->buf_bytes, h->buf_bytes, h->stream));
    if (nbuf == 1) {
        // B_n = collide(pull(B_{n-1}) + wall rule): the step this handle would have taken
        CK(h, launch_step(step_launch(h, 0, h->stream), h->coef));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    h->cur = 1;
    h->t = hd.t;
    h->snap_valid = 0;
    return LBM_OK;
}

int lbm_query(lbm_handle h, long* t, int* status) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    int st = 0;
    CK(h, cudaMemcpyAsync(&st, h->status_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (t) *t = h->t;
    if (status) *status = st ? LBM_ERR_DIVERGED : LBM_OK;
    return LBM_OK;
}

int lbm_destroy(lbm_handle h) {
    if (!h) return LBM_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    free_handle(h);
    if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e));
    return LBM_OK;
}

const char* lbm_last_error(lbm_handle h) { return h ? h->err.c_str() : g_init_error.c_str(); }

}  // extern "C"
