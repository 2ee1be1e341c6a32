// C ABI of the optical-flow solver: handle, workspace, the mixed-precision
// PCG driver, adaptation and adjoint entry points.  Declarations and the
// contract of every entry point are in include/of.h.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "of.h"
#include "of_launch.h"
#include "of_schwarz.cuh"
#include "of_schwarz_h2.cuh"

using ofk::PairDesc;
using ofk::PairScalars;

constexpr long long kDefaultWaitLimit = 4000000000LL;  // about 2 s at 2 GHz

struct of_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // grid
    int batch = 0;
    of_grid_opts opts{};
    ofl::SmoothTaps taps{};      // K_sigma (r = 0: none)
    ofl::SmoothTaps taps_rho{};  // K_rho (r = 0: none)
    void* eld = nullptr;         // K_rho element data: 18 planes of frame_elems values (rho > 0)
    void* eldg = nullptr;        // K_rho adjoint work, same layout
    // adaptation-pass VJP work (allocated on first use)
    double *vjp_w = nullptr, *vjp_buf = nullptr, *vjp_part = nullptr;
    unsigned long long* vjp_argmax = nullptr;
    int fp64 = 1;
    size_t es = 8;  // storage element size (frames, alpha, inner vectors)
    std::vector<PairDesc> pd;
    std::vector<int4> blocks, tiles;
    std::vector<int> blk0, nblk, tile0, ntile;
    long long frame_elems = 0, vec_elems = 0, pair_elems = 0;
    int nblk_total = 0, ntiles_total = 0, rows_per_block = 16;
    // device memory
    std::vector<void*> allocs;
    size_t alloc_bytes = 0, alloc_limit = 0;  // bytes held; test hook: budget (0: none)
    bool setup_started = false;               // of_setup_grid got past validation (workspace released)
    void *f1 = nullptr, *f2 = nullptr, *alpha = nullptr, *eta = nullptr;
    void* lamel = nullptr;  // per-element lambda [H][pitch][2] (grid option lambda_min > 0), else null
    double *x[2] = {nullptr, nullptr}, *usol = nullptr, *cvec = nullptr;
    void *r = nullptr, *z = nullptr, *q = nullptr, *d = nullptr, *p0 = nullptr, *p1 = nullptr;
    PairDesc* pd_dev = nullptr;
    int4 *blocks_dev = nullptr, *tiles_dev = nullptr;
    CUtensorMap* tmaps_dev = nullptr;
    uint32_t* ntab_dev = nullptr;
    int sch_threads = 0, sch_npt = 1, sch_grid = 1, sch_nstage = 2;
    void *cell0 = nullptr, *cell1 = nullptr;  // preconditioner element records [H][pitch]
    int h2 = 0;                                // FP16 paired sweeps (mixed path)
    void *cp0 = nullptr, *cp1 = nullptr;       // their paired records [H][pitch] (16 bytes each)
    bool cells_dirty = true;
    // inner PCG loop as a CUDA graph: while(any pair iterating) { apply; Schwarz }
    cudaGraph_t loop_graph = nullptr;
    cudaGraphExec_t loop_exec = nullptr;
    long long spin_limit = kDefaultWaitLimit;  // bound of every device wait, clock64 cycles
    // two-level preconditioner (coarse space)
    std::vector<ofl::CoarsePair> cps;
    ofl::CoarseBufs coarse{};

    int starve_bytes = 0;                      // test hook: staging waits expect this much more
    cudaGraphConditionalHandle loop_cond = 0;
    PairScalars* sc_dev = nullptr;
    PairScalars* sc_host = nullptr;  // pinned
    double *partA = nullptr, *partS = nullptr, *etamax = nullptr;
    unsigned *cntA = nullptr, *cntS = nullptr;
    int* err_dev = nullptr;
    void* staging = nullptr;
    size_t staging_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // kernel timing (of_set_profiling)
    struct ProfRec { int kind; cudaEvent_t a, b; };
    bool prof = false;
    std::vector<cudaEvent_t> evpool;
    std::vector<ProfRec> recs;
    of_profile ptot{};
    // state
    std::vector<char> frames_set, alpha_set;
    std::vector<std::vector<double>> ras_hist;  // stationary Schwarz: ||U^k - U^{k-1}|| per pair
    bool solved = false;
    of_solve_opts last_opts{};
};

static thread_local std::string g_create_err;

namespace {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

of_status fail(of_ctx* h, of_status s, const std::string& m) {
    if (h) h->err = m;
    else g_create_err = m;
    return s;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) {                                                                     \
            return fail(h, e_ == cudaErrorMemoryAllocation ? OF_ERR_OOM : OF_ERR_CUDA,               \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                         \
        }                                                                                            \
    } while (0)

// Device block of the pair scalars: [batch] PairScalars, the error word (16
// bytes), [batch] doubles of the stationary Schwarz history.
size_t sc_block_bytes(int batch) { return sizeof(PairScalars) * batch + 16 + sizeof(double) * batch; }
double* ras_hist_dev(of_ctx* h) {
    return reinterpret_cast<double*>(reinterpret_cast<char*>(h->sc_dev + h->batch) + 16);
}
const double* ras_hist_host(of_ctx* h) {
    return reinterpret_cast<const double*>(reinterpret_cast<const char*>(h->sc_host + h->batch) + 16);
}

// Reads the pair scalars, the device error word and the history slots back
// (one stream-ordered copy) and waits for it.  Returns the error word.
of_status read_scalars(of_ctx* h, cudaStream_t st, int* errw) {
    CK(cudaMemcpyAsync(h->sc_host, h->sc_dev, sc_block_bytes(h->batch), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *errw = *reinterpret_cast<const int*>(h->sc_host + h->batch);
    return OF_OK;
}

// Status of a nonzero device error word: bit 0 a bounded wait ran out, bit 2
// a device index check failed (bounds-check build only).
of_status err_status(of_ctx* h, int errw) {
    if (errw & ofk::OF_ERR_BIT_BOUNDS)
        return fail(h, OF_ERR_CUDA, "a device index check failed (library built with OF_BOUNDS_CHECK)");
    return fail(h, OF_ERR_TIMEOUT, "a bounded device wait (TMA staging) ran out");
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int tcode(of_dtype dt) { return dt == OF_F64 ? ofl::T_F64 : ofl::T_F32; }
size_t tsize(of_dtype dt) { return dt == OF_F64 ? 8 : 4; }

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

void free_all(of_ctx* h) {
    h->coarse = ofl::CoarseBufs{};
    h->cps.clear();
    if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
    if (h->loop_graph) cudaGraphDestroy(h->loop_graph);
    h->loop_exec = nullptr;
    h->loop_graph = nullptr;
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    h->alloc_bytes = 0;
    if (h->sc_host) cudaFreeHost(h->sc_host);
    h->sc_host = nullptr;
    h->f1 = h->f2 = h->alpha = h->eta = nullptr;
    h->lamel = nullptr;
    h->x[0] = h->x[1] = h->usol = h->cvec = nullptr;
    h->r = h->z = h->q = h->d = h->p0 = h->p1 = nullptr;
    h->batch = 0;
    h->solved = false;
    h->ras_hist.clear();
}

template <typename T>
cudaError_t dalloc(of_ctx* h, T** p, size_t bytes) {
    void* v = nullptr;
    if (bytes < 256) bytes = 256;
    if (h->alloc_limit && h->alloc_bytes + bytes > h->alloc_limit) return cudaErrorMemoryAllocation;  // injected
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e != cudaSuccess) return e;
    h->allocs.push_back(v);
    h->alloc_bytes += bytes;
    *p = (T*)v;
    return cudaSuccess;
}

// NVTX range over one entry point or phase (a no-op unless a tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

cudaEvent_t pool_event(of_ctx* h) {
    if (!h->evpool.empty()) {
        cudaEvent_t e = h->evpool.back();
        h->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch `fn` (returns cudaError_t), bracketed by events when profiling.
template <typename F>
cudaError_t timed(of_ctx* h, int kind, F fn) {
    if (!h->prof) {
        h->ptot.launches[kind] += 1;  // launches are counted always, timed only when profiling
        return fn();
    }
    cudaEvent_t a = pool_event(h), b = pool_event(h);
    cudaEventRecord(a, h->stream);
    cudaError_t e = fn();
    cudaEventRecord(b, h->stream);
    h->recs.push_back({kind, a, b});
    return e;
}

void count_other(of_ctx* h, int n) { h->ptot.launches[3] += n; }

// Accumulates recorded launches (the stream must have passed them).
void prof_flush(of_ctx* h) {
    for (auto& r : h->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) h->ptot.ms[r.kind] += ms;
        h->ptot.launches[r.kind] += 1;
        h->evpool.push_back(r.a);
        h->evpool.push_back(r.b);
    }
    h->recs.clear();
}

template <typename... A>
cudaError_t cp2d(of_ctx* h, A... a) {
    count_other(h, 1);
    return ofl::copy2d(a...);
}
template <typename... A>
cudaError_t fl2d(of_ctx* h, A... a) {
    count_other(h, 1);
    return ofl::fill2d(a...);
}

ofl::SolveBufs solve_bufs(of_ctx* h) {
    ofl::SolveBufs B;
    memset(&B, 0, sizeof(B));
    B.pairs = h->pd_dev;
    B.blocks = h->blocks_dev;
    B.tiles = h->tiles_dev;
    B.tmaps = h->tmaps_dev;
    B.ntab = h->ntab_dev;
    B.sch_threads = h->sch_threads;
    B.sch_npt = h->sch_npt;
    B.sch_grid = h->sch_grid;
    B.sch_nstage = h->sch_nstage;
    B.sc = h->sc_dev;
    B.partA = h->partA;
    B.partS = h->partS;
    B.cntA = h->cntA;
    B.cntS = h->cntS;
    B.err = h->err_dev;
    B.f1 = h->f1;
    B.f2 = h->f2;
    B.alpha = h->alpha;
    B.r = h->r;
    B.z = h->z;
    B.q = h->q;
    B.d = h->d;
    B.p0 = h->p0;
    B.p1 = h->p1;
    B.nblk = h->nblk_total;
    B.ntiles = h->ntiles_total;
    B.npairs = h->batch;
    B.rows_per_block = h->rows_per_block;
    B.Tx = h->opts.tile_x;
    B.Ty = h->opts.tile_y;
    B.ov = h->opts.overlap;
    B.sweeps = h->opts.sweeps;
    B.lam = h->opts.lambda;
    B.omega = h->opts.omega;
    B.gms = h->opts.model == OF_MODEL_CONSTANT ? 0.0 : 1.0;
    B.eld = h->eld;
    B.eld_stride = h->frame_elems;
    B.fp64 = h->fp64;
    B.spin_limit = h->spin_limit;
    B.tx_extra = h->starve_bytes;
    B.coarse = h->coarse;
    B.h2 = h->h2;
    B.lamel = h->lamel;
    B.cp0 = h->cp0;
    B.cp1 = h->cp1;
    return B;
}

ofl::AdaptBufs adapt_bufs(of_ctx* h) {
    ofl::AdaptBufs A;
    memset(&A, 0, sizeof(A));
    A.pairs = h->pd_dev;
    A.f1 = h->f1;
    A.f2 = h->f2;
    A.alpha = h->alpha;
    A.u = h->usol;
    A.lamel = h->lamel;
    A.u32 = h->fp64 ? nullptr : (const float*)h->z;  // filled by of_adapt_alpha (z is free after a solve)
    A.eta = h->eta;
    A.etamax = h->etamax;
    A.lam = h->opts.lambda;
    A.gms = h->opts.model == OF_MODEL_CONSTANT ? 0.0 : 1.0;
    A.eld = h->eld;
    A.eld_stride = h->frame_elems;
    A.eldg = h->eldg;
    A.taps_rho = &h->taps_rho;
    A.fp64 = h->fp64;
    return A;
}

of_status check_pair(of_ctx* h, int pair) {
    if (!h) return OF_ERR_ARG;
    if (h->batch == 0) return fail(h, OF_ERR_STATE, "of_setup_grid has not been called");
    if (pair < 0 || pair >= h->batch) return fail(h, OF_ERR_ARG, "pair index out of range");
    return OF_OK;
}

// Copy a user array (rows x cols, row pitch upitch, dtype dt, host or device)
// into a workspace array (dtype of the handle, row pitch wpitch).
of_status copy_in(of_ctx* h, const void* src, of_dtype dt, long long upitch, void* dst, long long wpitch,
                  long long rows, long long cols) {
    const int st = tcode(dt), wt = h->fp64 ? ofl::T_F64 : ofl::T_F32;
    if (is_device_ptr(src)) {
        CK(cp2d(h, src, st, upitch, dst, wt, wpitch, rows, cols, h->stream));
    } else {
        const size_t need = (size_t)rows * cols * tsize(dt);
        if (need > h->staging_bytes) return fail(h, OF_ERR_ARG, "host array larger than the staging buffer");
        CK(cudaMemcpy2DAsync(h->staging, cols * tsize(dt), src, upitch * tsize(dt), cols * tsize(dt), rows,
                             cudaMemcpyHostToDevice, h->stream));
        CK(cp2d(h, h->staging, st, cols, dst, wt, wpitch, rows, cols, h->stream));
    }
    return OF_OK;
}

// Copy a workspace array (type wt) out to a user array (dtype dt, contiguous
// rows x cols), host or device.
of_status copy_out(of_ctx* h, const void* src, int wt, long long wpitch, void* dst, of_dtype dt, long long rows,
                   long long cols) {
    const int dtc = tcode(dt);
    if (is_device_ptr(dst)) {
        CK(cp2d(h, src, wt, wpitch, dst, dtc, cols, rows, cols, h->stream));
    } else {
        const size_t need = (size_t)rows * cols * tsize(dt);
        if (need > h->staging_bytes) return fail(h, OF_ERR_ARG, "host array larger than the staging buffer");
        CK(cp2d(h, src, wt, wpitch, h->staging, dtc, cols, rows, cols, h->stream));
        CK(cudaMemcpyAsync(dst, h->staging, need, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));  // the staging buffer is reused by the next copy
    }
    return OF_OK;
}

of_status encode_maps(of_ctx* h) {
    auto enc = get_encode();
    if (!enc) return fail(h, OF_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const int Tx = h->opts.tile_x, Ty = h->opts.tile_y, ov = h->opts.overlap;
    const CUtensorMapDataType dtp = h->fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const size_t es = h->es;
    std::vector<CUtensorMap> maps((size_t)h->batch * ofk::TM_PER_PAIR);
    for (int p = 0; p < h->batch; ++p) {
        const PairDesc& d = h->pd[p];
        CUtensorMap* m = &maps[(size_t)p * ofk::TM_PER_PAIR];
        const cuuint32_t es1[3] = {1, 1, 1};
        {  // preconditioner cell records, viewed as 8-byte units: u units per record
            const int u = h->fp64 ? 4 : 1;
            const int RW = ofk::sch_rw(Tx, ov), RH = ofk::sch_rh(Ty, ov);
            const cuuint64_t dims[2] = {(cuuint64_t)d.W * u, (cuuint64_t)d.H};
            const cuuint64_t str[1] = {(cuuint64_t)d.pitch * u * 8};
            const cuuint32_t box[2] = {(cuuint32_t)(RW * u), (cuuint32_t)RH};
            for (int k = 0; k < 2; ++k) {
                char* base = (char*)(k == 0 ? h->cell0 : h->cell1) + d.frame_off * u * 8;
                CUresult rc = enc(&m[k == 0 ? ofk::TM_C0 : ofk::TM_C1], CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, dims,
                                  str, box, es1, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (rc != CUDA_SUCCESS) return fail(h, OF_ERR_CUDA, "tensor map (cells) encoding failed");
            }
        }
        if (h->h2) {  // paired records of the FP16 sweeps: 16 bytes = two 8-byte units per record
            const int RW = ofk::sch_rw(Tx, ov), HP = ofk::h2_hp(Ty, ov);
            // ov + 1 extra rows on top: a tile's box starts at row y0 >= 0 and
            // never in the fill region (whose lane-B half would be lost)
            const cuuint64_t dims[2] = {(cuuint64_t)d.W * 2, (cuuint64_t)(d.H + ov + 1)};
            const cuuint64_t str[1] = {(cuuint64_t)d.pitch * 16};
            const cuuint32_t box[2] = {(cuuint32_t)(RW * 2), (cuuint32_t)(HP + 1)};
            for (int k = 0; k < 2; ++k) {
                char* base = (char*)(k == 0 ? h->cp0 : h->cp1) + d.pair_off * 16;
                CUresult rc = enc(&m[k == 0 ? ofk::TM_P0 : ofk::TM_P1], CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, dims,
                                  str, box, es1, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (rc != CUDA_SUCCESS) return fail(h, OF_ERR_CUDA, "tensor map (paired records) encoding failed");
            }
        }
        {  // r and q planes
            const cuuint64_t dims[3] = {(cuuint64_t)d.W, (cuuint64_t)d.H, 3};
            const cuuint64_t str[2] = {(cuuint64_t)d.pitch * es, (cuuint64_t)d.H * d.pitch * es};
            const cuuint32_t box[3] = {(cuuint32_t)Tx, (cuuint32_t)Ty, 3};
            for (int k = 0; k < 3; ++k) {
                void* buf = k == 0 ? h->r : (k == 1 ? h->q : h->z);
                char* base = (char*)buf + d.vec_off * es;
                CUresult rc = enc(&m[k == 0 ? ofk::TM_R : (k == 1 ? ofk::TM_Q : ofk::TM_Z)], dtp, 3, base, dims, str, box, es1,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (rc != CUDA_SUCCESS) return fail(h, OF_ERR_CUDA, "tensor map (vectors) encoding failed");
            }
        }
    }
    CUtensorMap* dev = nullptr;
    CK(dalloc(h, &dev, maps.size() * sizeof(CUtensorMap)));
    CK(cudaMemcpyAsync(dev, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, h->stream));
    h->tmaps_dev = dev;
    return OF_OK;
}

constexpr int kLoopUnroll = 4;

// Builds the inner-loop graph: a while-node whose body is kLoopUnroll PCG
// iterations
// (apply, then Schwarz); the Schwarz kernel's last CTA sets the condition
// once no pair is iterating.  Returns false (and leaves no graph) if the
// driver cannot build it; the solve then polls from the host.
bool build_loop_graph(of_ctx* h) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraphConditionalHandle cond = 0;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    ok = ok && cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    alignas(cudaGraphNodeParams) unsigned char cp_buf[sizeof(cudaGraphNodeParams)] = {};
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_buf);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    ok = ok && cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ok = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            ofl::SolveBufs B = solve_bufs(h);
            B.use_cond = 1;
            B.cond = cond;
            // several iterations per check of the condition: iterations after a
            // pair has finished return at once (their kernels test its flag)
            cudaError_t e1 = cudaSuccess, e2 = cudaSuccess;
            for (int u = 0; u < kLoopUnroll; ++u) {
                B.use_cond = (u == kLoopUnroll - 1);  // only the last sets the condition
                if (e1 == cudaSuccess) e1 = ofl::launch_pcg_apply(B, cs);
                if (e2 == cudaSuccess) e2 = ofl::launch_pcg_precond(B, cs);
            }
            cudaGraph_t out = nullptr;
            cudaError_t e3 = cudaStreamEndCapture(cs, &out);
            ok = e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess;
        }
    }
    ok = ok && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (cs) cudaStreamDestroy(cs);
    if (!ok) {
        if (ex) cudaGraphExecDestroy(ex);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return false;
    }
    h->loop_graph = g;
    h->loop_exec = ex;
    h->loop_cond = cond;
    return true;
}

// The loop graph captures the kernels' parameters: rebuild it after they change.
of_status rebuild_loop_graph(of_ctx* h) {
    if (!h->loop_exec) return OF_OK;  // no grid yet, or the host loop is in use
    CK(cudaStreamSynchronize(h->stream));
    cudaGraphExecDestroy(h->loop_exec);
    cudaGraphDestroy(h->loop_graph);
    h->loop_exec = nullptr;
    h->loop_graph = nullptr;
    build_loop_graph(h);  // on failure the solve polls from the host
    return OF_OK;
}

// Recomputes the preconditioner's element records if frames or alpha changed.
of_status refresh_cells(of_ctx* h) {
    if (!h->cells_dirty) return OF_OK;
    ofl::SolveBufs B = solve_bufs(h);
    const size_t rb = h->fp64 ? 32 : 8;
    for (int p = 0; p < h->batch; ++p) {
        const PairDesc& d = h->pd[p];
        CK(ofl::launch_cells(B, p, d.W, d.H, (char*)h->cell0, (char*)h->cell1, h->stream));
        count_other(h, 1);
        (void)rb;
    }
    if (h->coarse.on) {
        // A_0 = R_0 A R_0^T (dense, banded), its band Cholesky factor and the
        // dense inverse
        const size_t es = h->fp64 ? 8 : 4;
        const ofl::CoarsePair& last = h->cps.back();
        CK(cudaMemsetAsync(h->coarse.Amat, 0, (size_t)(last.moff + (long long)last.n0 * last.n0) * es, h->stream));
        CK(ofl::launch_coarse_assemble(B, h->stream));
        count_other(h, 2);
        for (int p = 0; p < h->batch; ++p) {
            CK(ofl::launch_coarse_factor(B, p, h->cps[p].n0, h->cps[p].nx, h->cps[p].moff, h->stream));
            count_other(h, 3);
        }
        std::vector<int> info(h->batch);
        CK(cudaMemcpyAsync(info.data(), h->coarse.info, sizeof(int) * info.size(), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int v : info)
            if (v != 0) return fail(h, OF_ERR_BREAKDOWN, "coarse operator not positive definite");
    }
    h->cells_dirty = false;
    return OF_OK;
}

// The solve driver shared by of_solve and of_adjoint.  rhs == NULL: b from
// the frames; otherwise the FP64 right-hand side planes.  On return x[cur]
// holds the solution.
of_status run_solve(of_ctx* h, const of_solve_opts& o, const double* rhs, int* cur_out, std::vector<int>& passes_out) {
    of_status cs = refresh_cells(h);
    if (cs != OF_OK) return cs;
    ofl::SolveBufs B = solve_bufs(h);
    cudaStream_t st = h->stream;
    int cur = 0;
    // host-driven loop: poll every 8 iterations; when timing kernels, after
    // every iteration so that no launch past convergence enters the averages
    const int chunk = h->prof ? 1 : 8;
    int errw = 0;  // device error word, read back with the scalars
    passes_out.assign(h->batch, 0);
    CK(cudaMemsetAsync(h->cntA, 0, sizeof(unsigned) * (h->batch + h->nblk_total), st));
    CK(cudaMemsetAsync(h->cntS, 0, sizeof(unsigned) * h->batch, st));
    CK(cudaMemsetAsync(h->sc_dev, 0, sizeof(PairScalars) * h->batch, st));
    CK(cudaMemsetAsync(h->err_dev, 0, sizeof(int), st));
    for (int pass = 0;; ++pass) {
        NvtxRange nv_pass("refinement pass");
        const int first = (pass == 0);
        double* xout = first ? nullptr : h->x[1 - cur];
        // a cold start (x = 0) needs only the load vector for its first residual
        const double* xin = (first && !o.warm_start) ? nullptr : h->x[cur];
        CK(timed(h, 2, [&] { return ofl::launch_residual(B, xin, xout, rhs, first, o.rtol, o.inner_rtol, o.pass_frac, o.max_inner, st); }));
        if (!first) cur = 1 - cur;
        if (pass == o.max_outer) {
            of_status rs = read_scalars(h, st, &errw);
            if (rs != OF_OK) return rs;
            break;
        }
        CK(timed(h, 1, [&] { return ofl::launch_precond_first(B, st); }));
        if (h->loop_exec && !h->prof && !o.host_loop) {
            // the whole inner loop on the device; one read-back per pass
            CK(cudaGraphLaunch(h->loop_exec, st));
            of_status rs = read_scalars(h, st, &errw);
            if (rs != OF_OK) return rs;
            int body = 0;  // loop iterations = the most iterations any pair took in this pass
            for (int p = 0; p < h->batch; ++p) body = std::max(body, h->sc_host[p].it);
            body = (body + kLoopUnroll - 1) / kLoopUnroll * kLoopUnroll;  // whole bodies run
            h->ptot.launches[0] += body;
            h->ptot.launches[1] += body;
        } else {
            int it = 0;
            bool all_done = false;
            while (!all_done) {
                for (int c = 0; c < chunk; ++c, ++it) {
                    CK(timed(h, 0, [&] { return ofl::launch_pcg_apply(B, st); }));
                    CK(timed(h, 1, [&] { return ofl::launch_pcg_precond(B, st); }));
                }
                of_status rs = read_scalars(h, st, &errw);
                if (rs != OF_OK) return rs;
                all_done = true;
                for (int p = 0; p < h->batch; ++p) all_done = all_done && h->sc_host[p].done;
                if (errw) all_done = true;  // a bounded wait ran out: stop launching
                if (it >= o.max_inner + chunk) all_done = true;
            }
        }
        if (errw) break;  // a bounded wait ran out in this pass: no further launches
        bool all_conv = true;
        for (int p = 0; p < h->batch; ++p) {
            const bool conv = h->sc_host[p].pad[0] != 0;
            const bool broke = h->sc_host[p].status == 6 && h->sc_host[p].it == 0 && !conv;
            if (!conv && !broke) {
                all_conv = false;
                passes_out[p] = pass + 1;
            }
        }
        if (all_conv) break;
    }
    *cur_out = cur;
    prof_flush(h);
    if (errw) return err_status(h, errw);
    return OF_OK;
}

// The stationary Schwarz iteration (grid option schwarz = 1): residual
// (which folds the previous correction d into x), local solves, history.
// The residual kernel stops a pair whose residual is <= rtol ||b||; its
// later corrections are zero.  On return x[cur] holds the last iterate.
of_status run_ras(of_ctx* h, const of_solve_opts& o, int* cur_out, std::vector<int>& iters_out) {
    of_status cs = refresh_cells(h);
    if (cs != OF_OK) return cs;
    ofl::SolveBufs B = solve_bufs(h);
    cudaStream_t st = h->stream;
    int cur = 0, errw = 0;
    iters_out.assign(h->batch, 0);
    h->ras_hist.assign(h->batch, std::vector<double>());
    CK(cudaMemsetAsync(h->cntA, 0, sizeof(unsigned) * (h->batch + h->nblk_total), st));
    CK(cudaMemsetAsync(h->sc_dev, 0, sc_block_bytes(h->batch), st));
    for (int k = 0;; ++k) {
        NvtxRange nv_it("Schwarz iteration");
        const int first = (k == 0);
        double* xout = first ? nullptr : h->x[1 - cur];
        const double* xin = (first && !o.warm_start) ? nullptr : h->x[cur];
        CK(timed(h, 2, [&] { return ofl::launch_residual(B, xin, xout, nullptr, first, o.rtol, o.inner_rtol, o.pass_frac, 1, st); }));
        if (!first) cur = 1 - cur;
        of_status rs = read_scalars(h, st, &errw);
        if (rs != OF_OK) return rs;
        bool all_conv = true;
        for (int p = 0; p < h->batch; ++p) all_conv = all_conv && h->sc_host[p].pad[0] != 0;
        if (all_conv || k == o.max_inner) break;
        CK(ofl::launch_ras(B, h->cell0, h->cell1, ras_hist_dev(h), st));
        count_other(h, 2);
        rs = read_scalars(h, st, &errw);
        if (rs != OF_OK) return rs;
        const double* hv = ras_hist_host(h);
        for (int p = 0; p < h->batch; ++p)
            if (!h->sc_host[p].pad[0]) {
                h->ras_hist[p].push_back(hv[p]);
                iters_out[p] = k + 1;
            }
    }
    *cur_out = cur;
    prof_flush(h);
    if (errw) return err_status(h, errw);
    return OF_OK;
}

void fill_info(of_ctx* h, const std::vector<int>& passes, float ms, of_solve_info* info, of_status* worst) {
    *worst = OF_OK;
    for (int p = 0; p < h->batch; ++p) {
        const PairScalars& s = h->sc_host[p];
        of_status st = OF_OK;
        if (s.pad[0]) st = OF_OK;
        else if (s.status == 6 || !std::isfinite(s.res2)) st = OF_ERR_BREAKDOWN;
        else st = OF_ERR_NOT_CONVERGED;
        if (st == OF_ERR_BREAKDOWN || (st == OF_ERR_NOT_CONVERGED && *worst == OF_OK)) *worst = st;
        if (info) {
            info[p].status = st;
            info[p].outer_iters = passes[p];
            info[p].inner_iters = s.it_total;
            info[p].rel_residual = s.bnorm2 > 0 ? std::sqrt(s.res2 / s.bnorm2) : std::sqrt(s.res2);
            info[p].ms = ms;
        }
    }
}

of_solve_opts with_defaults(const of_solve_opts* o, int fp64) {
    of_solve_opts r{};
    if (o) r = *o;
    if (r.rtol <= 0) r.rtol = 1e-6;
    if (r.max_outer <= 0) r.max_outer = 20;
    if (r.max_inner <= 0) r.max_inner = 2000;
    // mixed: a pass may ask the FP32 PCG for a 5e-7 reduction, a little below
    // what FP32 arithmetic reaches in the true residual, so that the second pass
    // has little left to do; with passes aiming at half the outer tolerance this
    // ends near 0.3 rtol, which on the 3840x2160 layered pair keeps the flow
    // within 6e-5 px of the exact discrete solution at rtol 1e-6 (48 PCG
    // iterations; a 1e-6 floor: 46 iterations but 1.04e-4 px)
    if (r.inner_rtol <= 0) r.inner_rtol = fp64 ? 1e-12 : 5e-7;
    if (!(r.pass_frac > 0) || r.pass_frac > 1) r.pass_frac = 0.5;
    return r;
}

}  // namespace

extern "C" {

of_status of_create(of_handle* hp, int device, void* cuda_stream) {
    if (!hp) return fail(nullptr, OF_ERR_ARG, "null handle pointer");
    *hp = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(nullptr, OF_ERR_CUDA, "no CUDA device");
    }
    if (device < 0 || device >= n) return fail(nullptr, OF_ERR_ARG, "device out of range");
    of_ctx* h = new of_ctx();
    h->device = device;
    h->stream = (cudaStream_t)cuda_stream;
    DevGuard g(device);
    if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
        delete h;
        return fail(nullptr, OF_ERR_CUDA, "event creation failed");
    }
    *hp = h;
    return OF_OK;
}

static of_status setup_grid_impl(of_handle h, int batch, const int32_t* W, const int32_t* H,
                                 const of_grid_opts* o) {
    if (!h) return OF_ERR_ARG;
    if (batch < 1 || !W || !H) return fail(h, OF_ERR_ARG, "batch must be >= 1 with W and H arrays");
    DevGuard g(h->device);
    of_grid_opts opt{};
    if (o) opt = *o;
    if (opt.precision != OF_PREC_FP64 && opt.precision != OF_PREC_MIXED) return fail(h, OF_ERR_ARG, "bad precision");
    if (opt.tile_x == 0) opt.tile_x = 32;
    if (opt.tile_y == 0) opt.tile_y = 32;
    if (opt.lambda == 0) opt.lambda = 1.0;
    if (opt.omega == 0) opt.omega = 1.0;
    if (opt.preconditioner == OF_PC_JACOBI) {
        opt.overlap = 0;
        opt.sweeps = 0;
    } else {
        if (opt.sweeps == 0) opt.sweeps = 1;
    }
    if (!(opt.lambda > 0)) return fail(h, OF_ERR_ARG, "lambda must be > 0");
    if (!(opt.omega > 0 && opt.omega < 2)) return fail(h, OF_ERR_ARG, "omega must be in (0, 2)");
    if (!(opt.sigma >= 0 && opt.sigma <= 16)) return fail(h, OF_ERR_ARG, "sigma must be in [0, 16]");
    if (!(opt.rho >= 0 && opt.rho <= 16)) return fail(h, OF_ERR_ARG, "rho must be in [0, 16]");
    if (opt.model != OF_MODEL_ILLUMINATION && opt.model != OF_MODEL_CONSTANT) return fail(h, OF_ERR_ARG, "bad model");
    if (opt.coarse < 0 || (opt.coarse > 0 && opt.coarse < 4)) return fail(h, OF_ERR_ARG, "coarse spacing must be 0 or >= 4");
    if (opt.tile_x < 4 || opt.tile_y < 4 || opt.tile_x % 4 || opt.tile_y % 4 || opt.tile_x > 256 || opt.tile_y > 256)
        return fail(h, OF_ERR_ARG, "tile sizes must be multiples of 4 in [4, 256]");
    if (opt.schwarz != 0 && opt.schwarz != 1) return fail(h, OF_ERR_ARG, "schwarz must be 0 or 1");
    if (!(opt.lambda_min >= 0) || (opt.lambda_min > 0 && !(opt.lambda_min <= opt.lambda)))
        return fail(h, OF_ERR_ARG, "lambda_min must be 0 (constant lambda) or in (0, lambda]");
    if (opt.lambda_min > 0 && opt.rho > 0)
        return fail(h, OF_ERR_ARG, "a per-element lambda needs rho = 0");
    if (opt.schwarz == 1 && (opt.preconditioner != OF_PC_SCHWARZ || opt.coarse != 0 || opt.rho != 0))
        return fail(h, OF_ERR_ARG, "the stationary Schwarz iteration needs the Schwarz settings, coarse = 0, rho = 0");
    if (opt.overlap < 0 || opt.overlap > 32 || opt.sweeps < 0 || opt.sweeps > (opt.schwarz ? 4096 : 64))
        return fail(h, OF_ERR_ARG, "overlap must be in [0, 32] and sweeps in [0, 64] ([0, 4096] with schwarz = 1)");
    if (ofk::sch_rw(opt.tile_x, opt.overlap) * (opt.precision == OF_PREC_FP64 ? 4 : 1) > 256 ||
        ofk::sch_rh(opt.tile_y, opt.overlap) > 256)
        return fail(h, OF_ERR_ARG, "tile + overlap too large for one staged window");
    for (int p = 0; p < batch; ++p)
        if (W[p] < 2 || H[p] < 2 || W[p] > (1 << 20) || H[p] > (1 << 20))
            return fail(h, OF_ERR_ARG, "every frame must be at least 2x2 and at most 2^20 per side");
    const int fp64 = opt.precision == OF_PREC_FP64;
    int smax = 0;
    CK(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    // two TMA stages (prefetch of the next subdomain) when they fit, else one
    int nstage = 2;
    size_t smem = ofl::schwarz_smem_bytes(fp64, opt.tile_x, opt.tile_y, opt.overlap, 2);
    if (smem > (size_t)smax) {
        nstage = 1;
        smem = ofl::schwarz_smem_bytes(fp64, opt.tile_x, opt.tile_y, opt.overlap, 1);
    }
    std::vector<uint32_t> ntab;
    int sch_threads = 0, sch_npt = 1;
    if (!ofl::schwarz_node_table(fp64, opt.tile_x, opt.tile_y, opt.overlap, ntab, sch_threads, sch_npt))
        return fail(h, OF_ERR_ARG, "extended tile too large for one CTA (more than 2 nodes per thread and colour)");
    if (smem > (size_t)smax) return fail(h, OF_ERR_ARG, "tile/overlap need more shared memory than one CTA has");
    if (opt.schwarz == 1 && ofl::ras_smem_bytes(fp64, opt.tile_x, opt.tile_y, opt.overlap) > (size_t)smax)
        return fail(h, OF_ERR_ARG, "tile/overlap need more shared memory than one CTA has");
    // FP16 paired sweeps on the mixed path: by default wherever the tile can be
    // paired (half the extended height a multiple of 3, one pair per thread)
    if (opt.half_sweeps < -1 || opt.half_sweeps > 1) return fail(h, OF_ERR_ARG, "half_sweeps must be -1, 0 or 1");
    std::vector<uint32_t> ntab_h2;
    int h2_threads = 0, nstage_h2 = 2;
    size_t smem_h2 = 0;
    bool h2 = false;
    if (!fp64 && opt.half_sweeps >= 0 && opt.preconditioner == OF_PC_SCHWARZ && opt.sweeps >= 1 && opt.schwarz == 0 &&
        ofl::schwarz_h2_node_table(opt.tile_x, opt.tile_y, opt.overlap, ntab_h2, h2_threads)) {
        smem_h2 = ofl::schwarz_h2_smem_bytes(opt.tile_x, opt.tile_y, opt.overlap, 2);
        if (smem_h2 > (size_t)smax) {
            nstage_h2 = 1;
            smem_h2 = ofl::schwarz_h2_smem_bytes(opt.tile_x, opt.tile_y, opt.overlap, 1);
        }
        h2 = smem_h2 <= (size_t)smax;
    }
    if (opt.half_sweeps == 1 && !h2)
        return fail(h, OF_ERR_ARG, "FP16 paired sweeps need the mixed path, the Schwarz preconditioner with sweeps >= 1 "
                                   "and an extended tile height of 6k nodes (k <= 8)");

    CK(cudaStreamSynchronize(h->stream));
    free_all(h);
    h->setup_started = true;
    h->opts = opt;
    // K_sigma / K_rho taps: w_k = exp(-k^2 / (2 s^2)), |k| <= ceil(3 s)
    auto make_taps = [](double sd) {
        ofl::SmoothTaps T{};
        if (sd > 0) {
            const int r = std::min((int)std::ceil(3.0 * sd), ofl::OF_SMOOTH_RMAX);
            T.r = r;
            T.cw[0] = 0.0;
            for (int j = 0; j <= 2 * r; ++j) {
                const double k = j - r;
                T.w[j] = std::exp(-k * k / (2.0 * sd * sd));
                T.cw[j + 1] = T.cw[j] + T.w[j];
            }
        }
        return T;
    };
    h->taps = make_taps(opt.sigma);
    h->taps_rho = make_taps(opt.rho);
    h->fp64 = fp64;
    h->es = fp64 ? 8 : 4;
    h->batch = batch;
    h->pd.assign(batch, PairDesc{});
    h->blocks.clear();
    h->tiles.clear();
    h->blk0.assign(batch, 0);
    h->nblk.assign(batch, 0);
    h->tile0.assign(batch, 0);
    h->ntile.assign(batch, 0);
    long long fo = 0, vo = 0, po = 0;
    size_t stage = 0;
    const int cols_per_block = 31 * 4;
    for (int p = 0; p < batch; ++p) {
        PairDesc& d = h->pd[p];
        d.W = W[p];
        d.H = H[p];
        d.pitch = (W[p] + 31) / 32 * 32;
        d.frame_off = fo;
        d.vec_off = vo;
        d.tiles_x = (W[p] + opt.tile_x - 1) / opt.tile_x;
        d.tiles_y = (H[p] + opt.tile_y - 1) / opt.tile_y;
        d.tile0 = (int)h->tiles.size();
        for (int ty = 0; ty < d.tiles_y; ++ty)
            for (int tx = 0; tx < d.tiles_x; ++tx) h->tiles.push_back(make_int4(p, tx, ty, (int)h->tiles.size()));
        const int bx = (W[p] + cols_per_block - 1) / cols_per_block;
        const int by = (H[p] + h->rows_per_block - 1) / h->rows_per_block;
        d.blk0 = (int)h->blocks.size();
        d.nblk = bx * by;
        for (int yb = 0; yb < by; ++yb)
            for (int xb = 0; xb < bx; ++xb) h->blocks.push_back(make_int4(p, xb, yb, (int)h->blocks.size()));
        h->blk0[p] = d.blk0;
        h->nblk[p] = d.nblk;
        h->tile0[p] = d.tile0;
        h->ntile[p] = d.tiles_x * d.tiles_y;
        d.pair_off = po;
        fo += (long long)H[p] * d.pitch;
        po += (long long)(H[p] + opt.overlap + 1) * d.pitch;
        vo += 3LL * H[p] * d.pitch;
        stage = std::max(stage, (size_t)3 * W[p] * H[p] * 8);
    }
    h->frame_elems = fo;
    h->pair_elems = po;
    h->vec_elems = vo;
    h->nblk_total = (int)h->blocks.size();
    h->ntiles_total = (int)h->tiles.size();
    const size_t es = h->es;
    CK(dalloc(h, &h->f1, fo * es));
    CK(dalloc(h, &h->f2, fo * es));
    h->eld = nullptr;
    h->eldg = nullptr;
    h->vjp_w = h->vjp_buf = h->vjp_part = nullptr;
    h->vjp_argmax = nullptr;
    if (opt.rho > 0) {
        CK(dalloc(h, &h->eld, 18 * fo * es));
        CK(dalloc(h, &h->eldg, 18 * fo * es));
    }
    CK(dalloc(h, &h->alpha, 2 * fo * es));
    if (opt.lambda_min > 0) CK(dalloc(h, &h->lamel, 2 * fo * es));
    CK(dalloc(h, &h->eta, 2 * fo * es));
    CK(dalloc(h, &h->cell0, fo * (h->fp64 ? 32 : 8)));
    CK(dalloc(h, &h->cell1, fo * (h->fp64 ? 32 : 8)));
    h->h2 = h2 ? 1 : 0;
    h->cp0 = h->cp1 = nullptr;
    if (h2) {
        CK(dalloc(h, &h->cp0, h->pair_elems * 16));
        CK(dalloc(h, &h->cp1, h->pair_elems * 16));
    }
    for (int k = 0; k < 2; ++k) CK(dalloc(h, &h->x[k], vo * sizeof(double)));
    CK(dalloc(h, &h->usol, vo * sizeof(double)));
    CK(dalloc(h, &h->cvec, vo * sizeof(double)));
    CK(dalloc(h, &h->r, vo * es));
    CK(dalloc(h, &h->z, vo * es));
    CK(dalloc(h, &h->q, vo * es));
    CK(dalloc(h, &h->d, vo * es));
    CK(dalloc(h, &h->p0, vo * es));
    CK(dalloc(h, &h->p1, vo * es));
    CK(dalloc(h, &h->pd_dev, sizeof(PairDesc) * batch));
    CK(dalloc(h, &h->blocks_dev, sizeof(int4) * h->blocks.size()));
    CK(dalloc(h, &h->tiles_dev, sizeof(int4) * h->tiles.size()));
    // the device error word sits right after the pair scalars, so that one
    // stream-ordered copy per refinement pass reads both back
    // and after it one double per pair for the stationary Schwarz iteration's
    // ||U^k - U^{k-1}||
    CK(dalloc(h, &h->sc_dev, sc_block_bytes(batch)));
    h->err_dev = reinterpret_cast<int*>(h->sc_dev + batch);
    CK(dalloc(h, &h->partA, sizeof(double) * 2 * h->blocks.size()));
    CK(dalloc(h, &h->partS, sizeof(double) * 2 * h->tiles.size()));
    CK(dalloc(h, &h->etamax, sizeof(double) * batch));
    // per pair, then per apply block (the group counters of the FP32 apply's reduction)
    CK(dalloc(h, &h->cntA, sizeof(unsigned) * (batch + h->nblk_total)));
    CK(dalloc(h, &h->cntS, sizeof(unsigned) * batch));
    CK(dalloc(h, &h->staging, stage));
    h->staging_bytes = stage;
    CK(cudaMallocHost((void**)&h->sc_host, sc_block_bytes(batch)));
    cudaStream_t st = h->stream;
    CK(cudaMemcpyAsync(h->pd_dev, h->pd.data(), sizeof(PairDesc) * batch, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->blocks_dev, h->blocks.data(), sizeof(int4) * h->blocks.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->tiles_dev, h->tiles.data(), sizeof(int4) * h->tiles.size(), cudaMemcpyHostToDevice, st));
    for (void* v : {(void*)h->x[0], (void*)h->x[1], (void*)h->usol, (void*)h->cvec})
        CK(cudaMemsetAsync(v, 0, vo * sizeof(double), st));
    for (void* v : {h->r, h->z, h->q, h->d, h->p0, h->p1}) CK(cudaMemsetAsync(v, 0, vo * es, st));
    CK(cudaMemsetAsync(h->f1, 0, fo * es, st));
    CK(cudaMemsetAsync(h->f2, 0, fo * es, st));
    CK(cudaMemsetAsync(h->alpha, 0, 2 * fo * es, st));
    if (h->lamel) CK(ofl::fill2d(h->lamel, fp64 ? ofl::T_F64 : ofl::T_F32, 2 * fo, 1, 2 * fo, opt.lambda, st));
    CK(cudaMemsetAsync(h->sc_dev, 0, sizeof(PairScalars) * batch, st));
    CK(cudaMemsetAsync(h->cntA, 0, sizeof(unsigned) * (batch + h->nblk_total), st));
    CK(cudaMemsetAsync(h->cntS, 0, sizeof(unsigned) * batch, st));
    CK(cudaMemsetAsync(h->err_dev, 0, sizeof(int), st));
    of_status s = encode_maps(h);
    if (s != OF_OK) return s;
    CK(dalloc(h, &h->ntab_dev, std::max(ntab.size(), ntab_h2.size()) * sizeof(uint32_t)));
    CK(cudaMemcpyAsync(h->ntab_dev, ntab.data(), ntab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    h->sch_threads = sch_threads;
    h->sch_npt = sch_npt;
    h->sch_nstage = nstage;
    CK(ofl::schwarz_configure(fp64, sch_npt, opt.tile_x, opt.tile_y, opt.overlap, smem));
    h->sch_grid = ofl::schwarz_max_grid(fp64, sch_npt, opt.tile_x, opt.tile_y, opt.overlap, sch_threads, smem);
    if (h2) {
        // the paired sweeps replace the FP32 sweeps of the PCG preconditioner
        CK(cudaMemcpyAsync(h->ntab_dev, ntab_h2.data(), ntab_h2.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        h->sch_threads = h2_threads;
        h->sch_npt = 1;
        h->sch_nstage = nstage_h2;
        CK(ofl::schwarz_h2_configure(opt.tile_x, opt.tile_y, opt.overlap, smem_h2));
        h->sch_grid = ofl::schwarz_h2_max_grid(opt.tile_x, opt.tile_y, opt.overlap, h2_threads, smem_h2);
    }
    if (opt.coarse > 0 && opt.preconditioner == OF_PC_SCHWARZ) {
        // coarse grid of every pair: nodes at 0, s, 2s, ... and W - 1 (same in y)
        std::vector<ofl::CoarseCell> cells;
        long long moff = 0, items = 0, boff = 0;
        int voff = 0, max_n0 = 0, max_nx = 0;
        h->cps.assign(batch, ofl::CoarsePair{});
        for (int p = 0; p < batch; ++p) {
            auto axis = [&](int n) {
                std::vector<int> v;
                for (int x = 0; x < n - 1; x += opt.coarse) v.push_back(x);
                v.push_back(n - 1);
                return v;
            };
            const std::vector<int> xs = axis(W[p]), ys = axis(H[p]);
            ofl::CoarsePair& cp = h->cps[p];
            cp.nx = (int)xs.size();
            cp.ny = (int)ys.size();
            cp.nc = cp.nx * cp.ny;
            cp.n0 = 3 * cp.nc;
            if (cp.n0 > 8192) return fail(h, OF_ERR_ARG, "coarse grid too fine: more than 8192 coarse unknowns per pair");
            cp.moff = moff;
            cp.boff = boff;
            cp.voff = voff;
            cp.cell0 = (int)cells.size();
            for (int l = 0; l + 1 < cp.ny; ++l)
                for (int k = 0; k + 1 < cp.nx; ++k) cells.push_back({p, k, l, xs[k], xs[k + 1], ys[l], ys[l + 1]});
            moff += (long long)cp.n0 * cp.n0;
            boff += (long long)cp.n0 * (3 * cp.nx + 6);
            voff += cp.n0;
            max_nx = std::max(max_nx, cp.nx);
            items += (long long)cp.nc * 81;
            max_n0 = std::max(max_n0, cp.n0);
        }
        ofl::CoarseBufs& C = h->coarse;
        const size_t ces = fp64 ? 8 : 4;
        ofl::CoarsePair* cps_dev = nullptr;
        ofl::CoarseCell* cells_dev = nullptr;
        CK(dalloc(h, &cps_dev, sizeof(ofl::CoarsePair) * batch));
        CK(dalloc(h, &cells_dev, sizeof(ofl::CoarseCell) * cells.size()));
        CK(cudaMemcpyAsync(cps_dev, h->cps.data(), sizeof(ofl::CoarsePair) * batch, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(cells_dev, cells.data(), sizeof(ofl::CoarseCell) * cells.size(), cudaMemcpyHostToDevice, st));
        C.cps = cps_dev;
        C.cells = cells_dev;
        C.ncells = (int)cells.size();
        C.scatter_items = items;
        if (3 * max_nx + 6 > (fp64 ? 160 : 230))
            return fail(h, OF_ERR_ARG, "coarse grid too wide: its band factorisation window does not fit in shared memory");
        char* blk = nullptr;
        char* Am = nullptr;
        char* Ai = nullptr;
        char* Lr = nullptr;
        char* Lc = nullptr;
        char* part = nullptr;
        char* yv = nullptr;
        CK(dalloc(h, &blk, cells.size() * 144 * ces));
        CK(dalloc(h, &Am, (size_t)moff * ces));
        CK(dalloc(h, &Ai, (size_t)moff * ces));
        CK(dalloc(h, &Lr, (size_t)boff * ces));
        CK(dalloc(h, &Lc, (size_t)boff * ces));
        CK(dalloc(h, &C.info, sizeof(int) * batch));
        CK(dalloc(h, &part, cells.size() * 12 * ces));
        CK(dalloc(h, &yv, (size_t)voff * ces));
        char* gv = nullptr;
        CK(dalloc(h, &gv, (size_t)voff * ces));
        C.g = gv;
        C.total_n0 = voff;
        CK(dalloc(h, &C.gy, sizeof(double) * voff));
        CK(dalloc(h, &C.cnt, sizeof(unsigned)));
        CK(cudaMemsetAsync(C.cnt, 0, sizeof(unsigned), st));
        C.blk = blk;
        C.Amat = Am;
        C.Ainv = Ai;
        C.Lr = Lr;
        C.Lc = Lc;
        C.part = part;
        C.y = yv;
        C.max_n0 = max_n0;
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        C.gemv_grid = std::max(1, std::min(8 * sms, (max_n0 + 7) / 8));  // one row per warp
        CK(ofl::coarse_configure(fp64, max_n0, max_nx));
        C.on = 1;
    }
    h->cells_dirty = true;
    h->frames_set.assign(batch, 0);
    h->alpha_set.assign(batch, 0);
    h->solved = false;
    CK(cudaStreamSynchronize(st));
    build_loop_graph(h);
    return OF_OK;
}

// A failure after validation leaves no grid (the old workspace is already
// released): later calls see OF_ERR_STATE instead of half-built buffers.
of_status of_setup_grid(of_handle h, int batch, const int32_t* W, const int32_t* H, const of_grid_opts* o) {
    if (!h) return OF_ERR_ARG;
    NvtxRange nv("of_setup_grid");
    h->setup_started = false;
    const of_status s = setup_grid_impl(h, batch, W, H, o);
    if (s != OF_OK && h->setup_started) free_all(h);
    return s;
}

of_status of_set_alloc_limit(of_handle h, int64_t bytes) {
    if (!h) return OF_ERR_ARG;
    if (bytes < 0) return fail(h, OF_ERR_ARG, "bytes must be >= 0");
    h->alloc_limit = (size_t)bytes;
    return OF_OK;
}

of_status of_set_frames(of_handle h, int pair, const void* f1, const void* f2, of_dtype dt, int64_t pitch) {
    NvtxRange nv("of_set_frames");
    of_status s = check_pair(h, pair);
    if (s != OF_OK) return s;
    const PairDesc& d = h->pd[pair];
    if (!f1 || !f2 || pitch < d.W) return fail(h, OF_ERR_ARG, "null frame or row pitch < W");
    DevGuard g(h->device);
    const size_t es = h->es;
    s = copy_in(h, f1, dt, pitch, (char*)h->f1 + d.frame_off * es, d.pitch, d.H, d.W);
    if (s != OF_OK) return s;
    s = copy_in(h, f2, dt, pitch, (char*)h->f2 + d.frame_off * es, d.pitch, d.H, d.W);
    if (s != OF_OK) return s;
    if (h->opts.sigma > 0) {  // f = K_sigma * I; the r vector of the pair is scratch here
        const int ty = h->fp64 ? ofl::T_F64 : ofl::T_F32;
        void* scratch = (char*)h->r + d.vec_off * es;
        CK(ofl::launch_smooth((char*)h->f1 + d.frame_off * es, scratch, ty, d.W, d.H, d.pitch, h->taps, false,
                              h->stream));
        CK(ofl::launch_smooth((char*)h->f2 + d.frame_off * es, scratch, ty, d.W, d.H, d.pitch, h->taps, false,
                              h->stream));
        count_other(h, 4);
    }
    if (h->eld) {  // K_rho element data from the stored frames
        const int ty = h->fp64 ? ofl::T_F64 : ofl::T_F32;
        void* scratch = (char*)h->r + d.vec_off * es;
        CK(ofl::launch_element_data((char*)h->f1 + d.frame_off * es, (char*)h->f2 + d.frame_off * es, ty, d.W, d.H,
                                    d.pitch, h->opts.model == OF_MODEL_CONSTANT ? 0.0 : 1.0,
                                    (char*)h->eld + d.frame_off * es, h->frame_elems, scratch, h->taps_rho,
                                    h->stream));
        count_other(h, 1 + 2 * 18);
    }
    h->frames_set[pair] = 1;
    h->solved = false;
    h->cells_dirty = true;
    return OF_OK;
}

of_status of_get_element_data(of_handle h, int pair, void* out, of_dtype dt) {
    of_status s = check_pair(h, pair);
    if (s != OF_OK) return s;
    if (!out) return fail(h, OF_ERR_ARG, "null output");
    if (!h->eld) return fail(h, OF_ERR_STATE, "no element data (rho = 0)");
    if (!h->frames_set[pair]) return fail(h, OF_ERR_STATE, "frames not set");
    DevGuard g(h->device);
    const PairDesc& d = h->pd[pair];
    const int ty = h->fp64 ? ofl::T_F64 : ofl::T_F32;
    const size_t oes = dt == OF_F64 ? 8 : 4;
    const long long plane = (long long)(d.H - 1) * (d.W - 1);
    for (int q = 0; q < 18; ++q) {
        s = copy_out(h, (char*)h->eld + ((long long)q * h->frame_elems + d.frame_off) * h->es, ty, d.pitch,
                     (char*)out + (size_t)q * plane * oes, dt, d.H - 1, d.W - 1);
        if (s != OF_OK) return s;
    }
    CK(cudaStreamSynchronize(h->stream));
    return OF_OK;
}

of_status of_get_frames(of_handle h, int pair, void* f1, void* f2, of_dtype dt) {
    of_status s = check_pair(h, pair);
    if (s != OF_OK) return s;
    if (!f1 || !f2) return fail(h, OF_ERR_ARG, "null frame");
    if (!h->frames_set[pair]) return fail(h, OF_ERR_STATE, "frames not set");
    DevGuard g(h->device);
    const PairDesc& d = h->pd[pair];
    const int ty = h->fp64 ? ofl::T_F64 : ofl::T_F32;
    s = copy_out(h, (char*)h->f1 + d.frame_off * h->es, ty, d.pitch, f1, dt, d.H, d.W);
    if (s != OF_OK) return s;
    s = copy_out(h, (char*)h->f2 + d.frame_off * h->es, ty, d.pitch, f2, dt, d.H, d.W);
    if (s != OF_OK) return s;
    CK(cudaStreamSynchronize(h->stream));
    return OF_OK;
}

of_status of_set_alpha(of_handle h, int pair, const void* alpha, double alpha_const, of_dtype dt) {
    of_status s = check_pair(h, pair);
    if (s != OF_OK) return s;
    const PairDesc& d = h->pd[pair];
    DevGuard g(h->device);
    void* dst = (char*)h->alpha + 2 * d.frame_off * h->es;
    if (!alpha) {
        if (!(alpha_const > 0) || !std::isfinite(alpha_const)) return fail(h, OF_ERR_ARG, "alpha_const must be > 0");
        CK(fl2d(h, dst, h->fp64 ? ofl::T_F64 : ofl::T_F32, 2LL * d.pitch, d.H - 1, 2LL * (d.W - 1), alpha_const,
                       h->stream));
    } else {
        s = copy_in(h, alpha, dt, 2LL * (d.W - 1), dst, 2LL * d.pitch, d.H - 1, 2LL * (d.W - 1));
        if (s != OF_OK) return s;
    }
    h->alpha_set[pair] = 1;
    h->solved = false;
    h->cells_dirty = true;
    return OF_OK;
}

of_status of_set_lambda(of_handle h, int pair, const void* lam, double lam_const, of_dtype dt) {
    of_status s = check_pair(h, pair);
    if (s != OF_OK) return s;
    if (!h->lamel) return fail(h, OF_ERR_STATE, "the grid has a constant lambda (lambda_min = 0)");
    const PairDesc& d = h->pd[pair];
    DevGuard g(h->device);
    void* dst = (char*)h->lamel + 2 * d.frame_off * h->es;
    if (!lam) {
        if (!(lam_const > 0) || !std::isfinite(lam_const)) return fail(h, OF_ERR_ARG, "lam_const must be > 0");
        CK(fl2d(h, dst, h->fp64 ? ofl::T_F64 : ofl::T_F32, 2LL * d.pitch, d.H - 1, 2LL * (d.W - 1), lam_const,
                h->stream));
    } else {
        s = copy_in(h, lam, dt, 2LL * (d.W - 1), dst, 2LL * d.pitch, d.H - 1, 2LL * (d.W - 1));
        if (s != OF_OK) return s;
    }
    h->solved = false;
    return OF_OK;
}

of_status of_get_lambda(of_handle h, int pair, void* lam, of_dtype dt) {
    of_status s = check_pair(h, pair);
    if (s != OF_OK) return s;
    if (!lam) return fail(h, OF_ERR_ARG, "null lambda");
    if (!h->lamel) return fail(h, OF_ERR_STATE, "the grid has a constant lambda (lambda_min = 0)");
    const PairDesc& d = h->pd[pair];
    DevGuard g(h->device);
    return copy_out(h, (char*)h->lamel + 2 * d.frame_off * h->es, h->fp64 ? ofl::T_F64 : ofl::T_F32, 2LL * d.pitch,
                    lam, dt, d.H - 1, 2LL * (d.W - 1));
}

of_status of_get_alpha(of_handle h, int pair, void* alpha, of_dtype dt) {
    of_status s = check_pair(h, pair);
    if (s != OF_OK) return s;
    if (!alpha) return fail(h, OF_ERR_ARG, "null alpha");
    const PairDesc& d = h->pd[pair];
    DevGuard g(h->device);
    return copy_out(h, (char*)h->alpha + 2 * d.frame_off * h->es, h->fp64 ? ofl::T_F64 : ofl::T_F32, 2LL * d.pitch,
                    alpha, dt, d.H - 1, 2LL * (d.W - 1));
}

of_status of_solve(of_handle h, const of_solve_opts* o, void* const* U, of_dtype dt, of_solve_info* info) {
    NvtxRange nv("of_solve");
    if (!h) return OF_ERR_ARG;
    if (h->batch == 0) return fail(h, OF_ERR_STATE, "of_setup_grid has not been called");
    for (int p = 0; p < h->batch; ++p)
        if (!h->frames_set[p] || !h->alpha_set[p]) return fail(h, OF_ERR_STATE, "frames or alpha not set for a pair");
    if (!U) return fail(h, OF_ERR_ARG, "null solution array list");
    for (int p = 0; p < h->batch; ++p)
        if (!U[p]) return fail(h, OF_ERR_ARG, "null solution array");
    DevGuard g(h->device);
    const of_solve_opts opt = with_defaults(o, h->fp64);
    cudaStream_t st = h->stream;
    CK(cudaEventRecord(h->ev0, st));
    for (int p = 0; p < h->batch; ++p) {
        const PairDesc& d = h->pd[p];
        double* x0 = h->x[0] + d.vec_off;
        if (opt.warm_start) {
            // [3][H][W] user planes -> [3][H][pitch] FP64 planes
            if (is_device_ptr(U[p])) {
                CK(cp2d(h, U[p], tcode(dt), d.W, x0, ofl::T_F64, d.pitch, 3LL * d.H, d.W, st));
            } else {
                CK(cudaMemcpyAsync(h->staging, U[p], 3ULL * d.H * d.W * tsize(dt), cudaMemcpyHostToDevice, st));
                CK(cp2d(h, h->staging, tcode(dt), d.W, x0, ofl::T_F64, d.pitch, 3LL * d.H, d.W, st));
            }
        } else {
            CK(cudaMemsetAsync(x0, 0, 3ULL * d.H * d.pitch * sizeof(double), st));
        }
    }
    int cur = 0;
    std::vector<int> passes;
    const bool ras = h->opts.schwarz == 1;
    h->ras_hist.clear();
    of_status s = ras ? run_ras(h, opt, &cur, passes) : run_solve(h, opt, nullptr, &cur, passes);
    if (s != OF_OK) return s;
    // the solution becomes the kept one by exchanging the buffers (the next
    // solve rewrites its iterate buffers before reading them; no graph holds them)
    std::swap(h->usol, h->x[cur]);
    for (int p = 0; p < h->batch; ++p) {
        const PairDesc& d = h->pd[p];
        s = copy_out(h, h->usol + d.vec_off, ofl::T_F64, d.pitch, U[p], dt, 3LL * d.H, d.W);
        if (s != OF_OK) return s;
    }
    CK(cudaEventRecord(h->ev1, st));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    of_status worst;
    fill_info(h, passes, ms, info, &worst);
    if (ras && info)
        for (int p = 0; p < h->batch; ++p) {
            info[p].outer_iters = 0;
            info[p].inner_iters = passes[p];
        }
    h->solved = true;
    h->last_opts = opt;
    if (worst != OF_OK) return fail(h, worst, worst == OF_ERR_BREAKDOWN ? "CG breakdown (singular or indefinite data)"
                                                                       : "not converged within the iteration caps");
    return OF_OK;
}

of_status of_adapt_alpha(of_handle h, double kappa, double eta_thr, double alpha_th, void* const* eta, of_dtype dt) {
    NvtxRange nv("of_adapt_alpha");
    if (!h) return OF_ERR_ARG;
    if (!h->solved) return fail(h, OF_ERR_STATE, "of_adapt_alpha needs a previous of_solve");
    if (!(kappa >= 0) || !(alpha_th > 0)) return fail(h, OF_ERR_ARG, "kappa must be >= 0 and alpha_th > 0");
    DevGuard g(h->device);
    ofl::AdaptBufs A = adapt_bufs(h);
    cudaStream_t st = h->stream;
    CK(cudaMemsetAsync(h->etamax, 0, sizeof(double) * h->batch, st));
    for (int p = 0; p < h->batch; ++p) {
        const PairDesc& d = h->pd[p];
        if (!h->fp64)  // the FP32 path's indicator reads an FP32 copy of the solution
            CK(cp2d(h, h->usol + d.vec_off, ofl::T_F64, d.pitch, (float*)h->z + d.vec_off, ofl::T_F32, d.pitch,
                    3LL * d.H, d.W, st));
        CK(ofl::launch_indicator(A, p, d.H, d.W, st));
        count_other(h, 1);
        if (eta && eta[p]) {
            of_status s = copy_out(h, (char*)h->eta + 2 * d.frame_off * h->es, h->fp64 ? ofl::T_F64 : ofl::T_F32,
                                   2LL * d.pitch, eta[p], dt, d.H - 1, 2LL * (d.W - 1));
            if (s != OF_OK) return s;
        }
        CK(ofl::launch_alpha_update(A, p, d.H, d.W, kappa, eta_thr, alpha_th, st));
        count_other(h, 1);
        if (h->lamel) {  // the per-element lambda by the same rule, with its own threshold
            CK(ofl::launch_alpha_update(A, p, d.H, d.W, kappa, eta_thr, h->opts.lambda_min, st, h->lamel));
            count_other(h, 1);
        }
    }
    CK(cudaStreamSynchronize(st));
    h->solved = false;  // alpha changed: the stored solution no longer belongs to it
    h->cells_dirty = true;
    return OF_OK;
}

of_status of_adapt_alpha_vjp(of_handle h, double kappa, double eta_thr, double alpha_th, void* const* dLdalpha_new,
                             void* const* dLdalpha, void* const* dLdU, void* const* dLdf2, void* const* dLdf1,
                             of_dtype dt) {
    if (h && h->lamel)
        return fail(h, OF_ERR_STATE, "the adaptation-pass VJP is not provided with a per-element lambda (lambda_min > 0)");
    NvtxRange nv("of_adapt_alpha_vjp");
    if (!h) return OF_ERR_ARG;
    if (!h->solved) return fail(h, OF_ERR_STATE, "of_adapt_alpha_vjp needs a previous of_solve at the current alpha");
    if (!(kappa >= 0) || !(alpha_th > 0)) return fail(h, OF_ERR_ARG, "kappa must be >= 0 and alpha_th > 0");
    if (!dLdalpha_new || !dLdalpha || !dLdU) return fail(h, OF_ERR_ARG, "null dL/dalpha_new, dL/dalpha or dL/dU list");
    for (int p = 0; p < h->batch; ++p) {
        void* arr[5] = {dLdalpha_new[p], dLdalpha[p], dLdU[p], dLdf2 ? dLdf2[p] : nullptr, dLdf1 ? dLdf1[p] : nullptr};
        for (int k = 0; k < 5; ++k) {
            if (k < 3 && !arr[k]) return fail(h, OF_ERR_ARG, "null array");
            if (arr[k] && !is_device_ptr(arr[k])) return fail(h, OF_ERR_ARG, "of_adapt_alpha_vjp takes device arrays");
        }
    }
    DevGuard g(h->device);
    cudaStream_t st = h->stream;
    if (!h->vjp_w) {
        long long maxparts = 1;
        for (const PairDesc& d : h->pd) maxparts = std::max(maxparts, (long long)((d.W - 1 + 127) / 128) * (d.H - 1));
        CK(dalloc(h, &h->vjp_w, 2 * h->frame_elems * sizeof(double)));
        CK(dalloc(h, &h->vjp_buf, 26 * h->frame_elems * sizeof(double)));
        CK(dalloc(h, &h->vjp_part, maxparts * sizeof(double)));
        CK(dalloc(h, &h->vjp_argmax, sizeof(unsigned long long)));
    }
    ofl::AdaptBufs A = adapt_bufs(h);
    A.vjp_w = h->vjp_w;
    A.vjp_buf = h->vjp_buf;
    A.vjp_part = h->vjp_part;
    A.vjp_argmax = h->vjp_argmax;
    A.eld_stride = h->frame_elems;
    CK(cudaMemsetAsync(h->etamax, 0, sizeof(double) * h->batch, st));
    for (int p = 0; p < h->batch; ++p) {
        const PairDesc& d = h->pd[p];
        if (!h->fp64)  // the indicator of the forward pass reads an FP32 copy of the solution
            CK(cp2d(h, h->usol + d.vec_off, ofl::T_F64, d.pitch, (float*)h->z + d.vec_off, ofl::T_F32, d.pitch,
                    3LL * d.H, d.W, st));
        CK(ofl::launch_indicator(A, p, d.H, d.W, st));
        A.frame_off = d.frame_off;  // K_rho^T passes: the pair's planes, its r vector as scratch
        A.pitch = d.pitch;
        A.scratch = (char*)h->r + d.vec_off * h->es;
        CK(ofl::launch_adapt_vjp(A, p, d.H, d.W, kappa, eta_thr, alpha_th, dLdalpha_new[p], dLdalpha[p], dLdU[p],
                                 dLdf2 ? dLdf2[p] : nullptr, dLdf1 ? dLdf1[p] : nullptr, tcode(dt), st));
        count_other(h, 6 + (h->eld && (dLdf2 || dLdf1) ? 1 + 2 * 18 : 0));
        // with K_sigma the frame gradients are w.r.t. the images given to of_set_frames
        void* sscr = (char*)h->q + d.vec_off * h->es;
        for (void* fgrad : {dLdf2 ? dLdf2[p] : nullptr, dLdf1 ? dLdf1[p] : nullptr})
            if (fgrad && h->opts.sigma > 0)
                CK(ofl::launch_smooth(fgrad, sscr, tcode(dt), d.W, d.H, d.W, h->taps, true, st));
    }
    CK(cudaStreamSynchronize(st));
    return OF_OK;
}

of_status of_adjoint(of_handle h, void* const* dLdU, void* const* dLdalpha, void* const* dLdf2, void* const* dLdf1,
                     of_dtype dt, of_solve_info* info) {
    NvtxRange nv("of_adjoint");
    if (!h) return OF_ERR_ARG;
    if (!h->solved) return fail(h, OF_ERR_STATE, "of_adjoint needs a previous of_solve");
    if (!dLdU) return fail(h, OF_ERR_ARG, "null dL/dU list");
    DevGuard g(h->device);
    cudaStream_t st = h->stream;
    CK(cudaEventRecord(h->ev0, st));
    for (int p = 0; p < h->batch; ++p) {
        const PairDesc& d = h->pd[p];
        if (!dLdU[p]) return fail(h, OF_ERR_ARG, "null dL/dU array");
        double* c = h->cvec + d.vec_off;
        if (is_device_ptr(dLdU[p])) {
            CK(cp2d(h, dLdU[p], tcode(dt), d.W, c, ofl::T_F64, d.pitch, 3LL * d.H, d.W, st));
        } else {
            CK(cudaMemcpyAsync(h->staging, dLdU[p], 3ULL * d.H * d.W * tsize(dt), cudaMemcpyHostToDevice, st));
            CK(cp2d(h, h->staging, tcode(dt), d.W, c, ofl::T_F64, d.pitch, 3LL * d.H, d.W, st));
        }
        CK(cudaMemsetAsync(h->x[0] + d.vec_off, 0, 3ULL * d.H * d.pitch * sizeof(double), st));
    }
    of_solve_opts opt = h->last_opts;
    opt.warm_start = 0;  // the adjoint state starts from zero
    int cur = 0;
    std::vector<int> passes;
    of_status s = run_solve(h, opt, h->cvec, &cur, passes);
    if (s != OF_OK) return s;
    ofl::AdaptBufs A = adapt_bufs(h);
    for (int p = 0; p < h->batch; ++p) {
        const PairDesc& d = h->pd[p];
        A.frame_off = d.frame_off;  // K_rho^T passes: the pair's planes, its r vector as scratch
        A.pitch = d.pitch;
        A.scratch = (char*)h->r + d.vec_off * h->es;
        void* da = dLdalpha ? dLdalpha[p] : nullptr;
        void* d2 = dLdf2 ? dLdf2[p] : nullptr;
        void* d1 = dLdf1 ? dLdf1[p] : nullptr;
        // device outputs are written directly; host outputs go through the staging buffer
        const bool host_any = (da && !is_device_ptr(da)) || (d2 && !is_device_ptr(d2)) || (d1 && !is_device_ptr(d1));
        // with K_sigma, the frame gradients are taken w.r.t. the images I given to
        // of_set_frames: dL/dI = S^T dL/df (S = K_sigma), applied in place
        void* sscr = (char*)h->q + d.vec_off * h->es;  // H x W values of dt fit in the q planes
        auto smooth_t = [&](void* g) {
            return h->opts.sigma > 0 ? ofl::launch_smooth(g, sscr, tcode(dt), d.W, d.H, d.W, h->taps, true, st)
                                     : cudaSuccess;
        };
        if (!host_any) {
            CK(ofl::launch_adjoint_grad(A, p, d.H, d.W, h->x[cur], da, d2, d1, tcode(dt), st));
            if (d2) CK(smooth_t(d2));
            if (d1) CK(smooth_t(d1));
        } else {
            // one output at a time through the staging buffer
            const size_t esz = tsize(dt);
            struct Item { void* dst; int kind; size_t n; } items[3] = {
                {da, 0, (size_t)2 * (d.W - 1) * (d.H - 1)}, {d2, 1, (size_t)d.W * d.H}, {d1, 2, (size_t)d.W * d.H}};
            for (auto& it : items) {
                if (!it.dst) continue;
                if (is_device_ptr(it.dst)) {
                    CK(ofl::launch_adjoint_grad(A, p, d.H, d.W, h->x[cur], it.kind == 0 ? it.dst : nullptr,
                                                it.kind == 1 ? it.dst : nullptr, it.kind == 2 ? it.dst : nullptr,
                                                tcode(dt), st));
                    if (it.kind != 0) CK(smooth_t(it.dst));
                } else {
                    CK(ofl::launch_adjoint_grad(A, p, d.H, d.W, h->x[cur], it.kind == 0 ? h->staging : nullptr,
                                                it.kind == 1 ? h->staging : nullptr,
                                                it.kind == 2 ? h->staging : nullptr, tcode(dt), st));
                    if (it.kind != 0) CK(smooth_t(h->staging));
                    CK(cudaMemcpyAsync(it.dst, h->staging, it.n * esz, cudaMemcpyDeviceToHost, st));
                    CK(cudaStreamSynchronize(st));
                }
            }
        }
    }
    CK(cudaEventRecord(h->ev1, st));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    of_status worst;
    fill_info(h, passes, ms, info, &worst);
    if (worst != OF_OK) return fail(h, worst, "adjoint solve did not converge");
    return OF_OK;
}

of_status of_apply(of_handle h, int pair, const void* p, void* q, void* b, of_dtype dt) {
    of_status s = check_pair(h, pair);
    if (s != OF_OK) return s;
    if (!p || !q) return fail(h, OF_ERR_ARG, "null p or q");
    if (!h->frames_set[pair] || !h->alpha_set[pair]) return fail(h, OF_ERR_STATE, "frames or alpha not set");
    DevGuard g(h->device);
    const PairDesc& d = h->pd[pair];
    const size_t es = h->es;
    const int wt = h->fp64 ? ofl::T_F64 : ofl::T_F32;
    void* zin = (char*)h->z + d.vec_off * es;
    s = copy_in(h, p, dt, d.W, zin, d.pitch, 3LL * d.H, d.W);
    if (s != OF_OK) return s;
    ofl::SolveBufs B = solve_bufs(h);
    CK(cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream));
    CK(ofl::launch_apply(B, pair, h->blk0[pair], h->nblk[pair], h->z, h->q, b ? h->d : nullptr, h->stream));
    s = copy_out(h, (char*)h->q + d.vec_off * es, wt, d.pitch, q, dt, 3LL * d.H, d.W);
    if (s != OF_OK) return s;
    if (b) {
        s = copy_out(h, (char*)h->d + d.vec_off * es, wt, d.pitch, b, dt, 3LL * d.H, d.W);
        if (s != OF_OK) return s;
    }
    int errw = 0;
    s = read_scalars(h, h->stream, &errw);
    if (s != OF_OK) return s;
    if (errw) return err_status(h, errw);
    return OF_OK;
}

of_status of_precondition(of_handle h, int pair, const void* r, void* z, of_dtype dt) {
    of_status s = check_pair(h, pair);
    if (s != OF_OK) return s;
    if (!r || !z) return fail(h, OF_ERR_ARG, "null r or z");
    if (!h->frames_set[pair] || !h->alpha_set[pair]) return fail(h, OF_ERR_STATE, "frames or alpha not set");
    DevGuard g(h->device);
    const PairDesc& d = h->pd[pair];
    const size_t es = h->es;
    s = copy_in(h, r, dt, d.W, (char*)h->r + d.vec_off * es, d.pitch, 3LL * d.H, d.W);
    if (s != OF_OK) return s;
    s = refresh_cells(h);
    if (s != OF_OK) return s;
    ofl::SolveBufs B = solve_bufs(h);
    CK(cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream));
    CK(ofl::launch_precond_only(B, pair, h->tile0[pair], h->ntile[pair], h->stream));
    s = copy_out(h, (char*)h->z + d.vec_off * es, h->fp64 ? ofl::T_F64 : ofl::T_F32, d.pitch, z, dt, 3LL * d.H, d.W);
    if (s != OF_OK) return s;
    int errw = 0;
    s = read_scalars(h, h->stream, &errw);
    if (s != OF_OK) return s;
    if (errw) return err_status(h, errw);
    return OF_OK;
}

of_status of_residual(of_handle h, int pair, const void* U, of_dtype dt, double* rel) {
    of_status s = check_pair(h, pair);
    if (s != OF_OK) return s;
    if (!U || !rel) return fail(h, OF_ERR_ARG, "null U or result");
    if (!h->frames_set[pair] || !h->alpha_set[pair]) return fail(h, OF_ERR_STATE, "frames or alpha not set");
    DevGuard g(h->device);
    const PairDesc& d = h->pd[pair];
    cudaStream_t st = h->stream;
    double* c = h->cvec + d.vec_off;
    if (is_device_ptr(U)) {
        CK(cp2d(h, U, tcode(dt), d.W, c, ofl::T_F64, d.pitch, 3LL * d.H, d.W, st));
    } else {
        CK(cudaMemcpyAsync(h->staging, U, 3ULL * d.H * d.W * tsize(dt), cudaMemcpyHostToDevice, st));
        CK(cp2d(h, h->staging, tcode(dt), d.W, c, ofl::T_F64, d.pitch, 3LL * d.H, d.W, st));
    }
    ofl::SolveBufs B = solve_bufs(h);
    B.blocks = h->blocks_dev + h->blk0[pair];
    B.nblk = h->nblk[pair];
    CK(ofl::launch_residual(B, h->cvec, nullptr, nullptr, 1, 1e-300, 1e-300, 0.5, 1, st));
    PairScalars sc;
    CK(cudaMemcpyAsync(&sc, h->sc_dev + pair, sizeof(sc), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *rel = sc.bnorm2 > 0 ? std::sqrt(sc.res2 / sc.bnorm2) : std::sqrt(sc.res2);
    return OF_OK;
}

of_status of_get_schwarz_history(of_handle h, int pair, double* hist, int cap, int* n) {
    if (!h) return OF_ERR_ARG;
    if (pair < 0 || pair >= h->batch || !n || (cap > 0 && !hist)) return fail(h, OF_ERR_ARG, "bad pair or null output");
    if (h->ras_hist.size() != (size_t)h->batch)
        return fail(h, OF_ERR_STATE, "the last of_solve was not a stationary Schwarz solve");
    const std::vector<double>& v = h->ras_hist[pair];
    *n = (int)v.size();
    for (int i = 0; i < cap && i < (int)v.size(); ++i) hist[i] = v[i];
    return OF_OK;
}

of_status of_set_profiling(of_handle h, int on) {
    if (!h) return OF_ERR_ARG;
    h->prof = on != 0;
    h->ptot = of_profile{};
    return OF_OK;
}

of_status of_get_profile(of_handle h, of_profile* out) {
    if (!h || !out) return OF_ERR_ARG;
    DevGuard g(h->device);
    CK(cudaStreamSynchronize(h->stream));
    prof_flush(h);
    *out = h->ptot;
    h->ptot = of_profile{};
    return OF_OK;
}

of_status of_set_wait_limit(of_handle h, int64_t cycles) {
    if (!h) return OF_ERR_ARG;
    DevGuard g(h->device);
    h->spin_limit = cycles > 0 ? (long long)cycles : kDefaultWaitLimit;
    return rebuild_loop_graph(h);
}

of_status of_debug_starve_staging(of_handle h, int extra_bytes) {
    if (!h) return OF_ERR_ARG;
    if (extra_bytes < 0 || extra_bytes % 16 || extra_bytes > 4096)
        return fail(h, OF_ERR_ARG, "extra_bytes must be a multiple of 16 in [0, 4096]");
    DevGuard g(h->device);
    h->starve_bytes = extra_bytes;
    return rebuild_loop_graph(h);
}

of_status of_destroy(of_handle h) {
    if (!h) return OF_OK;
    {
        DevGuard g(h->device);
        cudaStreamSynchronize(h->stream);
        prof_flush(h);
        for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
        h->evpool.clear();
        free_all(h);
        if (h->ev0) cudaEventDestroy(h->ev0);
        if (h->ev1) cudaEventDestroy(h->ev1);
    }
    delete h;
    return OF_OK;
}

const char* of_last_error(of_handle h) {
    if (!h) return g_create_err.c_str();
    return h->err.c_str();
}

}  // extern "C"
