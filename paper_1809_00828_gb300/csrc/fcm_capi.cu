// extern "C" entry points of libfcm (declared in include/fcm.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "fcm_device.cuh"

using fcm::CgScalars;
using fcm::CgWork;

namespace {

thread_local std::string g_setup_error;
constexpr int kItersPerGraph = 8;

#define API_CUDA(C, call)                                                                              \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            (C)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                             \
            return e_ == cudaErrorMemoryAllocation ? FCM_ENOMEM : FCM_ECUDA;                           \
        }                                                                                              \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc((void **)p, sizeof(T) * std::max<size_t>(count, 1));
}

CgWork work_of(fcm_ctx *C)
{
    CgWork w;
    w.x = C->d_x;
    w.r = C->d_r;
    w.z = C->d_z;
    w.p = C->d_p;
    w.q = C->d_q;
    w.b = C->d_b;
    w.partial = C->d_partial;
    w.counter = C->d_counter;
    w.s = C->d_s;
    w.n = C->nlat;
    w.red_blocks = C->red_blocks;
    return w;
}

// The library works on its own stream; every call is ordered after the
// caller's stream on entry, and the caller's stream after the library's on exit.
struct StreamScope {
    fcm_ctx *C;
    explicit StreamScope(fcm_ctx *c) : C(c)
    {
        cudaEventRecord(C->ev_in, C->ustream);
        cudaStreamWaitEvent(C->stream, C->ev_in, 0);
    }
    ~StreamScope()
    {
        cudaEventRecord(C->ev_out, C->stream);
        cudaStreamWaitEvent(C->ustream, C->ev_out, 0);
    }
};

void apply_K_dev(fcm_ctx *C, const double *x, double *y, const int *done)
{
    fcm::launch_zero(y, C->nlat, done, C->stream);
    if (C->k_ff)
        fcm::launch_k_apply_ff(C->p, C->g, x, y, C->d_mask, C->d_elem_ff, C->kc, done, C->stream, C->ks);
    else
        fcm::launch_k_apply(C->p, C->g, x, y, C->d_mask, C->d_elem, C->kc, done, C->stream, C->ks);
}

void apply_S_dev(fcm_ctx *C, const double *r, double *z, const int *done)
{
    fcm::launch_schwarz_apply(C->p, C->g, r, z, C->d_f64, C->d_f32, C->plan, done, C->stream);
}

void destroy_graph(fcm_ctx *C)
{
    if (C->graph) cudaGraphExecDestroy(C->graph);
    C->graph = nullptr;
}

fcm_status build_graph(fcm_ctx *C)
{
    destroy_graph(C);
    const CgWork w = work_of(C);
    const int *done = &C->d_s->done;
    API_CUDA(C, cudaStreamBeginCapture(C->stream, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < kItersPerGraph; ++it) {
        apply_K_dev(C, C->d_p, C->d_q, done);
        fcm::cg_after_K(w, C->stream);
        apply_S_dev(C, C->d_r, C->d_z, done);
        fcm::cg_after_S(w, C->stream);
    }
    cudaGraph_t graph = nullptr;
    API_CUDA(C, cudaStreamEndCapture(C->stream, &graph));
    cudaError_t e = cudaGraphInstantiate(&C->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        C->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
        C->graph = nullptr;
        return FCM_ECUDA;
    }
    C->graph_iters = kItersPerGraph;
    return FCM_OK;
}

// One right-hand side, rhs and u on the device (rhs may alias the context's scratch vector).
fcm_status solve_one(fcm_ctx *C, const double *rhs, double tol, int maxit, double *u, fcm_solve_info &info)
{
    const CgWork w = work_of(C);
    cudaStream_t st = C->stream;
    fcm::launch_mask_copy(rhs, C->d_b, C->d_mask, C->nlat, st);
    fcm::cg_residual_norms(w, C->d_b, C->d_b, C->d_out2, st);
    double bb[2];
    API_CUDA(C, cudaMemcpyAsync(bb, C->d_out2, sizeof bb, cudaMemcpyDeviceToHost, st));
    API_CUDA(C, cudaStreamSynchronize(st));
    if (!std::isfinite(bb[1])) {
        C->err = "right-hand side has non-finite entries";
        return FCM_EINVAL;
    }
    CgScalars &h = *C->h_s;
    std::memset(&h, 0, sizeof h);
    h.tol = tol;
    h.maxit = maxit;
    API_CUDA(C, cudaMemcpyAsync(C->d_s, &h, sizeof h, cudaMemcpyHostToDevice, st));
    API_CUDA(C, cudaEventRecord(C->ev_t0, st));
    fcm::cg_init_kernels(w, st);
    apply_S_dev(C, C->d_r, C->d_z, nullptr);
    fcm::cg_after_first_S(w, st);
    API_CUDA(C, cudaGetLastError());
    if (!C->graph) {
        fcm_status s = build_graph(C);
        if (s != FCM_OK) return s;
    }
    bool timed_out = false;
    for (;;) {
        API_CUDA(C, cudaMemcpyAsync(&h, C->d_s, sizeof h, cudaMemcpyDeviceToHost, st));
        API_CUDA(C, cudaMemcpyAsync(C->h_err, C->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        API_CUDA(C, cudaStreamSynchronize(st));
        if (*C->h_err) {
            timed_out = true;  // a Schwarz apply gave up waiting for a factor copy: its z is wrong
            break;
        }
        if (h.done) break;
        API_CUDA(C, cudaGraphLaunch(C->graph, st));
    }
    API_CUDA(C, cudaEventRecord(C->ev_t1, st));
    API_CUDA(C, cudaMemcpyAsync(u, C->d_x, sizeof(double) * C->nlat, cudaMemcpyDeviceToDevice, st));
    // true residual ||b - K x|| / ||b||
    apply_K_dev(C, C->d_x, C->d_q, nullptr);
    fcm::cg_residual_norms(w, C->d_q, C->d_b, C->d_out2, st);
    API_CUDA(C, cudaMemcpyAsync(bb, C->d_out2, sizeof bb, cudaMemcpyDeviceToHost, st));
    API_CUDA(C, cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, C->ev_t0, C->ev_t1);
    info.iterations = h.it;
    info.relres = h.relres;
    info.true_relres = bb[1] > 0.0 ? std::sqrt(bb[0] / bb[1]) : 0.0;
    info.status = timed_out ? FCM_ETIMEOUT : h.status;
    info.seconds = ms * 1e-3;
    if (timed_out) {
        API_CUDA(C, cudaMemsetAsync(C->d_err, 0, sizeof(int), st));
        C->err = "a Schwarz apply gave up waiting for a factor copy (bounded mbarrier wait); the iterate is not valid";
    }
    return (fcm_status)info.status;
}

void free_ctx(fcm_ctx *C)
{
    if (!C) return;
    destroy_graph(C);
    void *ptrs[] = {C->d_elem, C->d_elem_ff, C->d_cell_elem, C->d_mask, C->d_rhs, C->d_cells, C->d_uncut, C->d_f64, C->d_f32,
                    C->d_slots, C->d_slot_of, C->d_items, C->d_zb, C->d_mzb, C->d_tc_tiles, C->d_tc_ft,
                    C->d_eta, C->d_jac, C->d_err,
                    C->d_x, C->d_r, C->d_z, C->d_p, C->d_q, C->d_b, C->d_t, C->d_partial, C->d_counter, C->d_s,
                    C->d_out2};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (C->h_s) cudaFreeHost(C->h_s);
    if (C->h_err) cudaFreeHost(C->h_err);
    if (C->d_m) cudaFree(C->d_m);
    if (C->d_ms) cudaFree(C->d_ms);
    if (C->h_ms) cudaFreeHost(C->h_ms);
    fcm::fcg_free(C->fcg);
    fcm::coarse_free(C->coarse);
    cudaEvent_t evs[] = {C->ev_in, C->ev_out, C->ev_t0, C->ev_t1, C->ev_f0, C->ev_f1, C->ev_fork, C->ev_join,
                         C->ks.fork, C->ks.join};
    for (auto e : evs)
        if (e) cudaEventDestroy(e);
    if (C->side) cudaStreamDestroy(C->side);
    if (C->ks.side) cudaStreamDestroy(C->ks.side);
    if (C->stream) cudaStreamDestroy(C->stream);
    delete C;
}

}  // namespace

// errors of calls without a context (set-up, U-Net) are reported by fcm_last_error(NULL)
std::string &fcm_unet_last_error() { return g_setup_error; }

namespace fcm {
void ctx_apply_K(fcm_ctx *C, const double *x, double *y) { apply_K_dev(C, x, y, nullptr); }
void ctx_apply_S(fcm_ctx *C, const double *r, double *z) { apply_S_dev(C, r, z, nullptr); }
void ctx_apply_K_flag(fcm_ctx *C, const double *x, double *y, const int *stop) { apply_K_dev(C, x, y, stop); }
void ctx_apply_S_flag(fcm_ctx *C, const double *r, double *z, const int *stop) { apply_S_dev(C, r, z, stop); }
fcm_status ctx_solve_one(fcm_ctx *C, const double *rhs, double tol, int maxit, double *u, fcm_solve_info &info)
{
    return solve_one(C, rhs, tol, maxit, u, info);
}
}  // namespace fcm

extern "C" {

fcm_status fcm_setup(const fcm_grid *grid, const fcm_geometry *geom, int p, double alpha, const fcm_bc *bc,
                     void *cuda_stream, fcm_ctx **out)
{
    if (!out || !grid || !geom || !bc) {
        g_setup_error = "fcm_setup: null argument";
        return FCM_EINVAL;
    }
    *out = nullptr;
    auto t0 = std::chrono::steady_clock::now();
    fcm_ctx *C = new (std::nothrow) fcm_ctx();
    if (!C) {
        g_setup_error = "fcm_setup: out of host memory";
        return FCM_ENOMEM;
    }
    std::string e;
    try {
        e = fcm::build_host_problem(*grid, *geom, p, alpha, *bc, C->hp);
    } catch (const std::bad_alloc &) {
        e = "out of host memory";
    } catch (...) {
        e = "host set-up failed";
    }
    if (!e.empty()) {
        g_setup_error = "fcm_setup: " + e;
        free_ctx(C);
        return e == "out of host memory" ? FCM_ENOMEM : FCM_EINVAL;
    }
    fcm::HostProblem &hp = C->hp;
    C->p = p;
    C->ne = hp.ne;
    C->nlat = hp.nlat;
    for (int a = 0; a < 3; ++a) {
        C->g.n[a] = hp.n[a];
        C->g.M[a] = hp.M[a];
    }
    C->ustream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&C->device);
    auto fail = [&](cudaError_t ce, const char *what) {
        g_setup_error = std::string("fcm_setup: ") + what + ": " + cudaGetErrorString(ce);
        free_ctx(C);
        return ce == cudaErrorMemoryAllocation ? FCM_ENOMEM : FCM_ECUDA;
    };
#define SETUP_CUDA(call)                          \
    do {                                          \
        cudaError_t ce_ = (call);                 \
        if (ce_ != cudaSuccess) return fail(ce_, #call); \
    } while (0)
    SETUP_CUDA(cudaStreamCreateWithFlags(&C->stream, cudaStreamNonBlocking));
    SETUP_CUDA(cudaEventCreateWithFlags(&C->ev_in, cudaEventDisableTiming));
    SETUP_CUDA(cudaEventCreateWithFlags(&C->ev_out, cudaEventDisableTiming));
    SETUP_CUDA(cudaEventCreate(&C->ev_t0));
    SETUP_CUDA(cudaEventCreate(&C->ev_t1));
    SETUP_CUDA(cudaEventCreate(&C->ev_f0));
    SETUP_CUDA(cudaEventCreate(&C->ev_f1));
    SETUP_CUDA(cudaStreamCreateWithFlags(&C->ks.side, cudaStreamNonBlocking));
    SETUP_CUDA(cudaEventCreateWithFlags(&C->ks.fork, cudaEventDisableTiming));
    SETUP_CUDA(cudaEventCreateWithFlags(&C->ks.join, cudaEventDisableTiming));
    const size_t ne2 = (size_t)hp.ne * hp.ne;
    const int64_t nelem = 1 + hp.ncut;
    SETUP_CUDA(dalloc(&C->d_elem, ne2 * nelem));
    SETUP_CUDA(dalloc(&C->d_cell_elem, hp.ncells));
    SETUP_CUDA(dalloc(&C->d_mask, hp.nlat));
    SETUP_CUDA(dalloc(&C->d_rhs, hp.nlat));
    SETUP_CUDA(dalloc(&C->d_eta, hp.ncells));
    cudaStream_t st = C->stream;
    SETUP_CUDA(cudaMemcpyAsync(C->d_elem, hp.Kref.data(), sizeof(double) * ne2, cudaMemcpyHostToDevice, st));
    if (hp.ncut > 0)
        SETUP_CUDA(cudaMemcpyAsync(C->d_elem + ne2, hp.Kcut.data(), sizeof(double) * ne2 * hp.ncut, cudaMemcpyHostToDevice, st));
    SETUP_CUDA(cudaMemcpyAsync(C->d_cell_elem, hp.cell_elem.data(), sizeof(int32_t) * hp.ncells, cudaMemcpyHostToDevice, st));
    SETUP_CUDA(cudaMemcpyAsync(C->d_mask, hp.mask.data(), hp.nlat, cudaMemcpyHostToDevice, st));
    SETUP_CUDA(cudaMemcpyAsync(C->d_rhs, hp.rhs.data(), sizeof(double) * hp.nlat, cudaMemcpyHostToDevice, st));
    {
        std::vector<float> eta_f(hp.eta.begin(), hp.eta.end());
        SETUP_CUDA(cudaMemcpyAsync(C->d_eta, eta_f.data(), sizeof(float) * hp.ncells, cudaMemcpyHostToDevice, st));
        SETUP_CUDA(cudaStreamSynchronize(st));
    }
    C->element_bytes = (int64_t)(sizeof(double) * ne2 * nelem);
    // active cells grouped by parity colour: uncut (matrix-free) and cut (own element matrix)
    std::vector<int2> cells;
    std::vector<int> uncut;
    cells.reserve(hp.ncut);
    uncut.reserve(hp.nactive);
    C->kc.cut_off[0] = 0;
    C->kc.uncut_off[0] = 0;
    for (int col = 0; col < 8; ++col) {
        for (int64_t ci = 0; ci < hp.ncells; ++ci) {
            if (hp.cell_elem[ci] < 0) continue;
            const int cx = (int)(ci % hp.n[0]), cy = (int)((ci / hp.n[0]) % hp.n[1]), cz = (int)(ci / ((int64_t)hp.n[0] * hp.n[1]));
            if ((cx & 1) + 2 * (cy & 1) + 4 * (cz & 1) != col) continue;
            if (hp.cell_elem[ci] == 0) uncut.push_back((int)ci);
            else cells.push_back(make_int2((int)ci, hp.cell_elem[ci]));
        }
        C->kc.cut_off[col + 1] = (int)cells.size();
        C->kc.uncut_off[col + 1] = (int)uncut.size();
    }
    SETUP_CUDA(dalloc(&C->d_cells, cells.size()));
    SETUP_CUDA(cudaMemcpyAsync(C->d_cells, cells.data(), sizeof(int2) * cells.size(), cudaMemcpyHostToDevice, st));
    SETUP_CUDA(dalloc(&C->d_uncut, uncut.size()));
    SETUP_CUDA(cudaMemcpyAsync(C->d_uncut, uncut.data(), sizeof(int) * uncut.size(), cudaMemcpyHostToDevice, st));
    C->kc.cut = C->d_cells;
    C->kc.uncut = C->d_uncut;
    fcm::make_sf_tables(hp, C->kc.sf);
    fcm::make_sf_tables_ff(C->kc.sf, C->kc.sff);
    // solver workspace
    double **vecs[] = {&C->d_x, &C->d_r, &C->d_z, &C->d_p, &C->d_q, &C->d_b, &C->d_t};
    for (double **v : vecs) {
        SETUP_CUDA(dalloc(v, hp.nlat));
        SETUP_CUDA(cudaMemsetAsync(*v, 0, sizeof(double) * hp.nlat, st));
    }
    int64_t rb = (hp.nlat + 255) / 256;
    C->red_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(rb, 152 * 8));
    SETUP_CUDA(dalloc(&C->d_partial, 2 * (size_t)C->red_blocks));
    SETUP_CUDA(dalloc(&C->d_counter, 1));
    SETUP_CUDA(cudaMemsetAsync(C->d_counter, 0, sizeof(unsigned), st));
    SETUP_CUDA(dalloc(&C->d_s, 1));
    SETUP_CUDA(cudaMemsetAsync(C->d_s, 0, sizeof(CgScalars), st));
    SETUP_CUDA(dalloc(&C->d_out2, 2));
    SETUP_CUDA(cudaMallocHost((void **)&C->h_s, sizeof(CgScalars)));
    SETUP_CUDA(cudaMallocHost((void **)&C->h_err, sizeof(int)));
    SETUP_CUDA(cudaStreamSynchronize(st));
#undef SETUP_CUDA
    // diagonal of K (Algorithm 1's diagonal scaling for DOFs in no block), then the element
    // matrices live on the device only
    hp.kdiag.assign(hp.nlat, 0.0);
    {
        const int q = hp.p + 1, ne = hp.ne;
        for (int64_t ci = 0; ci < hp.ncells; ++ci) {
            const int el = hp.cell_elem[ci];
            if (el < 0) continue;
            const double *Ke = el == 0 ? hp.Kref.data() : hp.Kcut.data() + (size_t)(el - 1) * ne * ne;
            const int cx = (int)(ci % hp.n[0]), cy = (int)((ci / hp.n[0]) % hp.n[1]),
                      cz = (int)(ci / ((int64_t)hp.n[0] * hp.n[1]));
            for (int iz = 0; iz < q; ++iz)
                for (int iy = 0; iy < q; ++iy)
                    for (int ix = 0; ix < q; ++ix) {
                        const int I = ix + q * (iy + q * iz);
                        const int64_t node = (hp.p * cx + ix) + (int64_t)hp.M[0] * ((hp.p * cy + iy) + (int64_t)hp.M[1] * (hp.p * cz + iz));
                        for (int a = 0; a < 3; ++a) hp.kdiag[3 * node + a] += Ke[(size_t)(3 * I + a) * ne + 3 * I + a];
                    }
        }
    }
    std::vector<double>().swap(hp.Kcut);
    C->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = C;
    return FCM_OK;
}

fcm_status fcm_info(const fcm_ctx *C, fcm_info_t *out)
{
    if (!C || !out) return FCM_EINVAL;
    const fcm::HostProblem &hp = C->hp;
    out->n_lattice = hp.nlat;
    out->n_free = hp.nfree;
    out->n_cells_active = hp.nactive;
    out->n_cells_cut = hp.ncut;
    out->n_patches = (int64_t)(hp.n[0] + 1) * (hp.n[1] + 1) * (hp.n[2] + 1);
    out->n_factors = C->n_factors;
    out->factor_bytes = C->factor_bytes;
    out->element_bytes = C->element_bytes;
    out->max_block = 3 * (2 * hp.p - 1) * (2 * hp.p - 1) * (2 * hp.p - 1);
    out->p = hp.p;
    out->setup_seconds = C->setup_seconds;
    out->precond_seconds = C->precond_seconds;
    out->n_blocks = C->n_blocks;
    out->n_blocks_fp32 = C->n_fp32_factors;
    {
        // cut cells: dense ne x ne; uncut cells: 3 components x (8 forward + 8 transposed) contractions of
        // Q^3 points x Q terms, plus ~21 multiply-adds of the stress per point
        const int64_t q = hp.p + 1;
        out->kapply_fmas = hp.ncut * (int64_t)hp.ne * hp.ne + (hp.nactive - hp.ncut) * (36 * q * q * q * q + 21 * q * q * q);
    }
    out->sapply_fmas = C->sapply_fmas;
    out->max_block_cond = C->max_cond;
    out->coarse_seconds = fcm::coarse_seconds(C->coarse);
    out->n_jacobi = C->n_jacobi;
    out->stream_rows = C->plan.rows;
    out->schwarz_concurrent = C->plan.concurrent;
    out->n_factors_ff = C->n_ff_factors;
    out->k_double_float = C->k_ff;
    {
        const fcm::SchwarzPlan &pl = C->plan;
        const bool tc = pl.n_tc_tiles > 0;
        const int own = (fcm::schwarz_uses_rows_kernel(C->p) ? pl.n_row_items : pl.n_col_items) > 0;
        out->s_apply_launches = C->have_precond ? (tc ? 1 : 0) + ((tc ? pl.n_tiles32_plain : pl.n_tiles32) > 0) +
                                                      (pl.n_tiles64 > 0) + own + 1
                                                : 0;
        int k = 1;  // zero y
        for (int c = 0; c < 8; ++c)
            k += (C->kc.uncut_off[c + 1] > C->kc.uncut_off[c]) + (C->kc.cut_off[c + 1] > C->kc.cut_off[c]);
        out->k_apply_launches = k;
    }
    out->n_gemm_blocks = C->n_gemm_blocks;
    for (int k = 0; k < 8; ++k) out->tune_seconds[k] = C->tune_seconds[k];
    out->device_error = 0;
    if (C->d_err) {
        int e = 0;
        if (cudaMemcpyAsync(&e, C->d_err, sizeof(int), cudaMemcpyDeviceToHost, C->stream) == cudaSuccess &&
            cudaStreamSynchronize(C->stream) == cudaSuccess)
            out->device_error = e;
    }
    return FCM_OK;
}

fcm_status fcm_rhs(const fcm_ctx *Cc, int load_case, double *b_dev)
{
    fcm_ctx *C = const_cast<fcm_ctx *>(Cc);
    if (!C || !b_dev) return FCM_EINVAL;
    if (load_case < 0 || load_case > 6) {
        C->err = "fcm_rhs: load case must be in 0..6";
        return FCM_EINVAL;
    }
    StreamScope sc(C);
    if (load_case == 0) {
        API_CUDA(C, cudaMemcpyAsync(b_dev, C->d_rhs, sizeof(double) * C->nlat, cudaMemcpyDeviceToDevice, C->stream));
    } else {
        // host copy of the set-up; synchronous so that the host buffer may be reused at once
        API_CUDA(C, cudaMemcpyAsync(b_dev, C->hp.rhs_strain.data() + (size_t)(load_case - 1) * C->nlat,
                                    sizeof(double) * C->nlat, cudaMemcpyHostToDevice, C->stream));
        API_CUDA(C, cudaStreamSynchronize(C->stream));
    }
    return FCM_OK;
}

fcm_status fcm_precond_build(fcm_ctx *C, const fcm_precond_opts *opts)
{
    if (!C) return FCM_EINVAL;
    fcm_precond_opts o;
    o.eps = 1e-13;
    o.precision = FCM_PREC_FP64;
    o.cond_fp64 = 1e7;
    o.block_rule = FCM_BLOCKS_VERTEX;
    o.eta_bar = 1.0;
    o.fixed_tiles = 0;
    o.simt_shared = 0;
    if (opts) o = *opts;
    if (!(o.eps == o.eps) || (o.precision != FCM_PREC_FP64 && o.precision != FCM_PREC_MIXED && o.precision != FCM_PREC_MIXED_FP64) || !(o.cond_fp64 > 0.0) ||
        (o.block_rule != FCM_BLOCKS_VERTEX && o.block_rule != FCM_BLOCKS_ELEMENT) ||
        (o.block_rule == FCM_BLOCKS_ELEMENT && !(o.eta_bar >= 0.0)) || o.fixed_tiles < 0 || o.fixed_tiles > 2 ||
        o.simt_shared < 0 || o.simt_shared > 1) {
        C->err = "fcm_precond_build: invalid options";
        return FCM_EINVAL;
    }
    StreamScope sc(C);
    // captured graphs hold the addresses of the plan and factor pools being replaced
    destroy_graph(C);
    fcm::fcg_forget_graph(C->fcg);
    C->have_precond = false;
    std::string e;
    try {
        e = fcm::build_preconditioner(C, o);
    } catch (const std::bad_alloc &) {
        e = "out of host memory";
    }
    if (!e.empty()) {
        C->err = "fcm_precond_build: " + e;
        return e.find("out of memory") != std::string::npos ? FCM_ENOMEM : FCM_ECUDA;
    }
    // address of fcm_apply_S_noalloc's static scratch on this context's device (looked up here, at
    // set-up and outside any capture, so that the allocation-free call itself only launches)
    C->noalloc_scratch = nullptr;
    C->noalloc_err.clear();
    int dev = -1;
    if (C->nlat > (int64_t)FCM_NOALLOC_MAX_LATTICE) {
        C->noalloc_err = "problem larger than FCM_NOALLOC_MAX_LATTICE";
    } else if (cudaGetDevice(&dev) != cudaSuccess || dev != C->device) {
        C->noalloc_err = "the context's device is not current";
    } else {
        const cudaError_t ce = fcm::noalloc_scratch_address(&C->noalloc_scratch);
        if (ce != cudaSuccess) C->noalloc_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ce);
    }
    return FCM_OK;
}

// nr independent PCG recurrences (one per right-hand side) that share every Schwarz launch: the block
// factors are read once per iteration for all nr residuals.  K is applied per right-hand side; each
// recurrence stops on its own ||S r|| / ||S b|| <= tol (its kernels then return at once).
static fcm_status solve_multi(fcm_ctx *C, const double *rhs, int nr, double tol, int maxit, double *u,
                              fcm_solve_info &agg)
{
    const int64_t n = C->nlat;
    cudaStream_t st = C->stream;
    if (C->m_nr != nr) {
        if (C->d_m) cudaFree(C->d_m);
        if (C->d_ms) cudaFree(C->d_ms);
        if (C->h_ms) cudaFreeHost(C->h_ms);
        if (C->d_mzb) cudaFree(C->d_mzb);
        C->d_m = nullptr;
        C->d_ms = nullptr;
        C->h_ms = nullptr;
        C->d_mzb = nullptr;
        C->m_nr = 0;
        API_CUDA(C, cudaMalloc(&C->d_m, sizeof(double) * 6 * (size_t)nr * n));
        API_CUDA(C, cudaMalloc(&C->d_ms, sizeof(CgScalars) * nr));
        API_CUDA(C, cudaMallocHost((void **)&C->h_ms, sizeof(CgScalars) * nr));
        API_CUDA(C, cudaMalloc(&C->d_mzb, sizeof(double) * (size_t)nr * C->plan.nslots * C->plan.zs));
        C->m_nr = nr;
    }
    double *X = C->d_m, *R = X + (size_t)nr * n, *Z = R + (size_t)nr * n, *Pd = Z + (size_t)nr * n,
           *Q = Pd + (size_t)nr * n, *B = Q + (size_t)nr * n;
    std::vector<CgWork> w(nr);
    double bb[2];
    for (int k = 0; k < nr; ++k) {
        w[k] = work_of(C);
        w[k].x = X + (size_t)k * n;
        w[k].r = R + (size_t)k * n;
        w[k].z = Z + (size_t)k * n;
        w[k].p = Pd + (size_t)k * n;
        w[k].q = Q + (size_t)k * n;
        w[k].b = B + (size_t)k * n;
        w[k].s = C->d_ms + k;
        fcm::launch_mask_copy(rhs + (size_t)k * n, w[k].b, C->d_mask, n, st);
        fcm::cg_residual_norms(w[k], w[k].b, w[k].b, C->d_out2, st);
        API_CUDA(C, cudaMemcpyAsync(bb, C->d_out2, sizeof bb, cudaMemcpyDeviceToHost, st));
        API_CUDA(C, cudaStreamSynchronize(st));
        if (!std::isfinite(bb[1])) {
            C->err = "right-hand side has non-finite entries";
            return FCM_EINVAL;
        }
        std::memset(C->h_ms + k, 0, sizeof(CgScalars));
        C->h_ms[k].tol = tol;
        C->h_ms[k].maxit = maxit;
    }
    API_CUDA(C, cudaMemcpyAsync(C->d_ms, C->h_ms, sizeof(CgScalars) * nr, cudaMemcpyHostToDevice, st));
    API_CUDA(C, cudaEventRecord(C->ev_t0, st));
    for (int k = 0; k < nr; ++k) fcm::cg_init_kernels(w[k], st);
    fcm::launch_schwarz_apply_multi(C->p, R, Z, n, nr, C->d_f64, C->d_f32, C->plan, C->d_mzb, nullptr, st);
    for (int k = 0; k < nr; ++k) fcm::cg_after_first_S(w[k], st);
    for (int it = 0;; ++it) {
        if (it % 8 == 0) {
            API_CUDA(C, cudaMemcpyAsync(C->h_ms, C->d_ms, sizeof(CgScalars) * nr, cudaMemcpyDeviceToHost, st));
            API_CUDA(C, cudaMemcpyAsync(C->h_err, C->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
            API_CUDA(C, cudaStreamSynchronize(st));
            if (*C->h_err) {
                API_CUDA(C, cudaMemsetAsync(C->d_err, 0, sizeof(int), st));
                C->err = "a Schwarz apply gave up waiting for a factor copy (bounded mbarrier wait); the iterates are not valid";
                agg.status = FCM_ETIMEOUT;
                return FCM_ETIMEOUT;
            }
            bool all = true;
            for (int k = 0; k < nr; ++k) all = all && C->h_ms[k].done;
            if (all) break;
        }
        for (int k = 0; k < nr; ++k) apply_K_dev(C, w[k].p, w[k].q, &C->d_ms[k].done);
        for (int k = 0; k < nr; ++k) fcm::cg_after_K(w[k], st);
        fcm::launch_schwarz_apply_multi(C->p, R, Z, n, nr, C->d_f64, C->d_f32, C->plan, C->d_mzb, nullptr, st);
        for (int k = 0; k < nr; ++k) fcm::cg_after_S(w[k], st);
        API_CUDA(C, cudaGetLastError());
    }
    API_CUDA(C, cudaEventRecord(C->ev_t1, st));
    API_CUDA(C, cudaMemcpyAsync(u, X, sizeof(double) * (size_t)nr * n, cudaMemcpyDeviceToDevice, st));
    fcm_status worst = FCM_OK;
    for (int k = 0; k < nr; ++k) {
        apply_K_dev(C, w[k].x, C->d_q, nullptr);
        fcm::cg_residual_norms(w[k], C->d_q, w[k].b, C->d_out2, st);
        API_CUDA(C, cudaMemcpyAsync(bb, C->d_out2, sizeof bb, cudaMemcpyDeviceToHost, st));
        API_CUDA(C, cudaStreamSynchronize(st));
        const CgScalars &h = C->h_ms[k];
        agg.iterations = std::max(agg.iterations, h.it);
        agg.relres = std::max(agg.relres, h.relres);
        agg.true_relres = std::max(agg.true_relres, bb[1] > 0.0 ? std::sqrt(bb[0] / bb[1]) : 0.0);
        if (h.status != FCM_OK && worst == FCM_OK) worst = (fcm_status)h.status;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, C->ev_t0, C->ev_t1);
    agg.seconds = ms * 1e-3;
    agg.status = worst;
    return worst;
}

static fcm_status solve_many(fcm_ctx *C, const double *rhs, int nrhs, double tol, int maxit, double *u, bool host,
                             int *iterations, double *final_relres)
{
    if (!C || !rhs || !u || nrhs < 1 || !(tol > 0.0) || maxit < 1) {
        if (C) C->err = "fcm_pcg_solve: invalid argument";
        return FCM_EINVAL;
    }
    if (!C->have_precond) {
        C->err = "fcm_pcg_solve: call fcm_precond_build first";
        return FCM_ESTATE;
    }
    StreamScope sc(C);
    // a failed wait of an earlier fcm_apply_S (reported by fcm_info) does not belong to this solve
    API_CUDA(C, cudaMemsetAsync(C->d_err, 0, sizeof(int), C->stream));
    fcm_solve_info agg = {};
    agg.status = FCM_OK;
    fcm_status worst = FCM_OK;
    const bool fp64_p4 = C->p == 4 && C->d_f64;
    if (!host && nrhs > 1 && nrhs <= 8 && !fp64_p4) {
        worst = solve_multi(C, rhs, nrhs, tol, maxit, u, agg);
        if (worst == FCM_EINVAL || worst == FCM_ECUDA || worst == FCM_ENOMEM || worst == FCM_ETIMEOUT) {
            agg.status = worst;
            C->last = agg;
            return worst;
        }
        nrhs = 0;  // done
    }
    for (int k = 0; k < nrhs; ++k) {
        const double *b = rhs + (size_t)k * C->nlat;
        double *x = u + (size_t)k * C->nlat;
        if (host) {
            API_CUDA(C, cudaMemcpyAsync(C->d_t, b, sizeof(double) * C->nlat, cudaMemcpyHostToDevice, C->stream));
            b = C->d_t;
        }
        fcm_solve_info one = {};
        fcm_status s = solve_one(C, b, tol, maxit, host ? C->d_t : x, one);
        if (host) {
            API_CUDA(C, cudaMemcpyAsync(x, C->d_t, sizeof(double) * C->nlat, cudaMemcpyDeviceToHost, C->stream));
            API_CUDA(C, cudaStreamSynchronize(C->stream));
        }
        if (s == FCM_EINVAL || s == FCM_ECUDA || s == FCM_ENOMEM) return s;
        if (s == FCM_ETIMEOUT) {
            C->last = one;
            return s;
        }
        agg.iterations = std::max(agg.iterations, one.iterations);
        agg.relres = std::max(agg.relres, one.relres);
        agg.true_relres = std::max(agg.true_relres, one.true_relres);
        agg.seconds += one.seconds;
        if (s != FCM_OK && worst == FCM_OK) worst = s;
    }
    agg.status = worst;
    C->last = agg;
    if (iterations) *iterations = agg.iterations;
    if (final_relres) *final_relres = agg.relres;
    if (worst == FCM_ENOTCONV) C->err = "fcm_pcg_solve: maxit reached";
    if (worst == FCM_EBREAKDOWN) C->err = "fcm_pcg_solve: CG breakdown (p^T K p <= 0 or non-finite scalar)";
    return worst;
}

fcm_status fcm_pcg_solve(fcm_ctx *C, const double *rhs_dev, int nrhs, double tol, int maxit, double *u_dev,
                         int *iterations, double *final_relres)
{
    return solve_many(C, rhs_dev, nrhs, tol, maxit, u_dev, false, iterations, final_relres);
}

fcm_status fcm_pcg_solve_host(fcm_ctx *C, const double *rhs_host, int nrhs, double tol, int maxit, double *u_host,
                              int *iterations, double *final_relres)
{
    return solve_many(C, rhs_host, nrhs, tol, maxit, u_host, true, iterations, final_relres);
}

fcm_status fcm_last_solve(const fcm_ctx *C, fcm_solve_info *out)
{
    if (!C || !out) return FCM_EINVAL;
    *out = C->last;
    return FCM_OK;
}

fcm_status fcm_apply_K(fcm_ctx *C, const double *x_dev, double *y_dev)
{
    if (!C || !x_dev || !y_dev) return FCM_EINVAL;
    StreamScope sc(C);
    fcm::launch_mask_copy(x_dev, C->d_t, C->d_mask, C->nlat, C->stream);
    apply_K_dev(C, C->d_t, y_dev, nullptr);
    API_CUDA(C, cudaGetLastError());
    return FCM_OK;
}

fcm_status fcm_apply_S(fcm_ctx *C, const double *r_dev, double *z_dev)
{
    if (!C || !r_dev || !z_dev) return FCM_EINVAL;
    if (!C->have_precond) {
        C->err = "fcm_apply_S: call fcm_precond_build first";
        return FCM_ESTATE;
    }
    StreamScope sc(C);
    fcm::launch_mask_copy(r_dev, C->d_t, C->d_mask, C->nlat, C->stream);
    apply_S_dev(C, C->d_t, z_dev, nullptr);
    API_CUDA(C, cudaGetLastError());
    return FCM_OK;
}

fcm_status fcm_apply_S_many(fcm_ctx *C, const double *r_dev, int nrhs, double *z_dev)
{
    if (!C || !r_dev || !z_dev || nrhs < 1 || nrhs > 8) {
        if (C) C->err = "fcm_apply_S_many: invalid argument (1 <= nrhs <= 8)";
        return FCM_EINVAL;
    }
    if (!C->have_precond) {
        C->err = "fcm_apply_S_many: call fcm_precond_build first";
        return FCM_ESTATE;
    }
    if (nrhs == 1) return fcm_apply_S(C, r_dev, z_dev);
    StreamScope sc(C);
    const int64_t n = C->nlat;
    if (C->m_nr != nrhs) {
        // the multi-RHS workspace of the solver, shaped for nrhs vectors
        if (C->d_m) cudaFree(C->d_m);
        if (C->d_ms) cudaFree(C->d_ms);
        if (C->h_ms) cudaFreeHost(C->h_ms);
        if (C->d_mzb) cudaFree(C->d_mzb);
        C->d_m = nullptr;
        C->d_ms = nullptr;
        C->h_ms = nullptr;
        C->d_mzb = nullptr;
        C->m_nr = 0;
        API_CUDA(C, cudaMalloc(&C->d_m, sizeof(double) * 6 * (size_t)nrhs * n));
        API_CUDA(C, cudaMalloc(&C->d_ms, sizeof(CgScalars) * nrhs));
        API_CUDA(C, cudaMallocHost((void **)&C->h_ms, sizeof(CgScalars) * nrhs));
        API_CUDA(C, cudaMalloc(&C->d_mzb, sizeof(double) * (size_t)nrhs * C->plan.nslots * C->plan.zs));
        C->m_nr = nrhs;
    }
    double *R = C->d_m;  // masked copies of the inputs
    for (int k = 0; k < nrhs; ++k) fcm::launch_mask_copy(r_dev + (size_t)k * n, R + (size_t)k * n, C->d_mask, n, C->stream);
    fcm::launch_schwarz_apply_multi(C->p, R, z_dev, n, nrhs, C->d_f64, C->d_f32, C->plan, C->d_mzb, nullptr, C->stream);
    API_CUDA(C, cudaGetLastError());
    return FCM_OK;
}

fcm_status fcm_set_k_precision(fcm_ctx *C, int mode)
{
    if (!C || (mode != FCM_K_FP64 && mode != FCM_K_DOUBLE_FLOAT)) {
        if (C) C->err = "fcm_set_k_precision: unknown mode";
        return FCM_EINVAL;
    }
    StreamScope sc(C);
    if (mode == FCM_K_DOUBLE_FLOAT && !C->d_elem_ff) {
        const int64_t n = C->element_bytes / (int64_t)sizeof(double);
        API_CUDA(C, cudaMalloc(&C->d_elem_ff, sizeof(float2) * (size_t)std::max<int64_t>(n, 1)));
        fcm::launch_to_ff_pairs(C->d_elem, C->d_elem_ff, n, C->stream);
        API_CUDA(C, cudaGetLastError());
        API_CUDA(C, cudaStreamSynchronize(C->stream));
    }
    if (C->k_ff != (mode == FCM_K_DOUBLE_FLOAT)) {
        C->k_ff = mode == FCM_K_DOUBLE_FLOAT;
        // the captured graphs hold the K launches of the other mode
        destroy_graph(C);
        fcm::fcg_forget_graph(C->fcg);
    }
    return FCM_OK;
}

fcm_status fcm_set_wait_limit(fcm_ctx *C, int tries)
{
    if (!C) return FCM_EINVAL;
    C->wait_tries = tries < 0 ? fcm::kWaitTries : tries;
    C->plan.wait_tries = C->wait_tries;
    // the captured graphs hold the plan's launch parameters
    destroy_graph(C);
    fcm::fcg_forget_graph(C->fcg);
    return FCM_OK;
}

const char *fcm_last_error(const fcm_ctx *C)
{
    return C ? C->err.c_str() : g_setup_error.c_str();
}

void fcm_destroy(fcm_ctx *C)
{
    if (!C) return;
    cudaStreamSynchronize(C->stream);
    free_ctx(C);
}

}  // extern "C"
