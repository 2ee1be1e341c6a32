// Host-side launch interface between the C ABI (of_api.cu) and the kernels
// (of_kernels.cu, of_adapt.cu).  Internal to the library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "of_common.cuh"

namespace ofl {

// element types of a copy
enum { T_F32 = 0, T_F64 = 1 };

// Strided 2D copy with conversion: dst[r*dpitch + c] = src[r*spitch + c].
cudaError_t copy2d(const void* src, int stype, long long spitch, void* dst, int dtype, long long dpitch,
                   long long rows, long long cols, cudaStream_t st);
// Fill rows x cols of a strided array with a constant.
cudaError_t fill2d(void* dst, int dtype, long long dpitch, long long rows, long long cols, double v, cudaStream_t st);

// Coarse space of the two-level preconditioner (of_coarse.cu)
struct CoarsePair {
    int nx, ny;      // coarse nodes in x and y (x = 0, s, 2s, ..., W - 1)
    int nc, n0;      // nodes, unknowns (3 nc, component-major)
    long long moff;  // offset of the pair's dense n0 x n0 matrices
    long long boff;  // offset of its band factors (n0 x (b+1), b = 3 nx + 5)
    int voff;        // offset of the pair's coarse vectors
    int cell0;       // first cell of the pair ((nx - 1) (ny - 1) cells, row-major)
};
struct CoarseCell {
    int pair, k, l;        // cell (k, l) of the pair
    int x0, x1, y0, y1;    // its corner coordinates (fine nodes)
};
struct CoarseBufs {
    int on;                   // 0: one-level preconditioner
    const CoarsePair* cps;    // [batch]
    const CoarseCell* cells;  // [ncells]
    int ncells;
    long long scatter_items;  // work items of the dense scatter
    void* blk;                // [ncells][144] cell blocks of A_0
    void* Amat;               // dense A_0 (column-major, per pair; node-major unknowns)
    void* Lr;                 // band Cholesky factor by rows and by columns
    void* Lc;
    int* info;                // [batch] factorisation status (0: positive definite)
    void* Ainv;               // dense A_0^{-1}
    void* part;               // [ncells][12] restriction partials
    void* g;                  // R_0 r
    void* y;                  // coarse correction
    double* gy;               // g_i y_i per coarse unknown
    int total_n0;             // coarse unknowns of the batch
    unsigned* cnt;            // arrival counter of the product kernel
    int max_n0, gemv_grid;
};
struct CoarseParams {
    const ofk::PairDesc* pairs;
    const CoarsePair* cps;
    int npairs;
    ofk::PairScalars* sc;
    const double* tpart;   // Schwarz per-subdomain partials (r.r, r.z_1)
    const void* Ainv;
    const void* part;
    void* g;
    void* y;
    double* gy;
    unsigned* counter;
    int* err;
    int first, apply_only, use_cond, only_pair;
    cudaGraphConditionalHandle cond;
};

struct SolveBufs {
    const ofk::PairDesc* pairs;
    const int4* blocks;
    const int4* tiles;
    const CUtensorMap* tmaps;
    const uint32_t* ntab;  // Schwarz thread -> node table (see schwarz_node_table)
    int sch_threads, sch_npt, sch_grid, sch_nstage;  // CTA size, nodes per thread and colour, grid, TMA stages
    ofk::PairScalars* sc;
    double* partA;
    double* partS;
    unsigned* cntA;
    unsigned* cntS;
    int* err;
    const void* f1;
    const void* f2;
    const void* alpha;
    void* r;
    void* z;
    void* q;
    void* d;
    void* p0;
    void* p1;
    int nblk, ntiles, rows_per_block, npairs;
    int Tx, Ty, ov, sweeps;
    double lam;
    double omega;  // relaxation factor of the local block SOR sweeps
    double gms;    // illumination column scale of the element data (1 or 0, see of_model)
    const void* eld;      // K_rho element data (18 planes, storage precision) or null (rho = 0)
    const void* lamel;    // per-element lambda [H][pitch][2] (storage precision) or null (constant)
    long long eld_stride; // plane stride of eld (elements)
    int fp64;            // 1: everything FP64; 0: FP32 inner with FP64 residual
    long long spin_limit;
    int use_cond;        // Schwarz launches inside the inner-loop graph set its condition
    int tx_extra;        // test hook: bytes the staging barriers expect beyond the copies
    CoarseBufs coarse;   // two-level preconditioner (coarse.on = 0: one level)
    int h2;              // mixed path: FP16 paired sweeps (of_schwarz_h2.cuh)
    void* cp0;           // their paired element records [H][pitch] (16 bytes each)
    void* cp1;
    cudaGraphConditionalHandle cond;
};

// Pass start: xout = xin + d + a p (unless first), r = rhs - A xout,
// ||r||^2, ||rhs||^2 (first) and the inner-pass set-up per pair.  xin = NULL
// means x = 0 (cold start): r = rhs, only the load is formed.
cudaError_t launch_residual(const SolveBufs& B, const double* xin, double* xout, const double* rhs_vec, int first,
                            double rtol, double inner_rtol, double pass_frac, int max_inner, cudaStream_t st);
// z = M r at the start of a pass (rz, rr, convergence check).
cudaError_t launch_precond_first(const SolveBufs& B, cudaStream_t st);
// One PCG iteration = launch_pcg_apply (p, d, q, a) then launch_pcg_precond
// (r, z, rz, beta, stop).
cudaError_t launch_pcg_apply(const SolveBufs& B, cudaStream_t st);
cudaError_t launch_pcg_precond(const SolveBufs& B, cudaStream_t st);
// Stand-alone operator apply (q = A p, optional b) in the inner precision
// (fp64 = 0: FP32) or FP64 for one pair (blocks of that pair only).
cudaError_t launch_apply(const SolveBufs& B, int pair, int blk0, int nblk, const void* p, void* q, void* b,
                         cudaStream_t st);
// Stand-alone preconditioner z = M r for one pair (tiles of that pair only);
// r must already be in B.r.
cudaError_t launch_precond_only(const SolveBufs& B, int pair, int tile0, int ntiles, cudaStream_t st);
size_t schwarz_smem_bytes(int fp64, int Tx, int Ty, int ov, int nstage);
// One stationary Schwarz iteration's local solves (of_ras.cu): d = sum_i
// R~_i^T A_i^{-1} R_i r over all tiles (B.r holds r), then per pair
// hist[p] = ||d||_2 and the scalars set so that the next residual launch
// folds d into x.  c0, c1: the element records.
cudaError_t launch_ras(const SolveBufs& B, const void* c0, const void* c1, double* hist, cudaStream_t st);
size_t ras_smem_bytes(int fp64, int Tx, int Ty, int ov);
// Cell records (element data of the preconditioner) of one pair, from the
// frames and alpha in the workspace; c0, c1: [H][pitch] records.
cudaError_t launch_cells(const SolveBufs& B, int pair, int W, int H, void* c0, void* c1, cudaStream_t st);
// Persistent CTAs of the Schwarz kernel that fit on the device at once.
int schwarz_max_grid(int fp64, int npt, int tx, int ty, int ov, int threads, size_t smem);
cudaError_t schwarz_configure(int fp64, int npt, int tx, int ty, int ov, size_t smem);
int schwarz_h2_max_grid(int tx, int ty, int ov, int threads, size_t smem);
cudaError_t schwarz_h2_configure(int tx, int ty, int ov, size_t smem);
// Host-built assignment of the extended tile's nodes to (colour, slot,
// thread) such that the 32 lanes of a warp touch 32 distinct shared-memory
// banks.  Returns false if a tile needs more than 2 slots per thread.
bool schwarz_node_table(int fp64, int Tx, int Ty, int ov, std::vector<uint32_t>& tab, int& threads, int& npt);
// The same for the FP16 paired sweeps: the node pairs (i, j), j < HP, of the
// extended tile, one pair per thread and colour, 32 distinct banks per warp.
// Returns false if the shape cannot be paired or needs more than 384 threads.
bool schwarz_h2_node_table(int Tx, int Ty, int ov, std::vector<uint32_t>& tab, int& threads);
size_t schwarz_h2_smem_bytes(int Tx, int Ty, int ov, int nstage);

// ---- adaptation (of_adapt.cu)
struct AdaptBufs {
    const ofk::PairDesc* pairs;
    const void* f1;
    const void* f2;
    void* alpha;
    const double* u;     // solution planes (FP64)
    const float* u32;    // FP32 copy of the solution planes (FP32 path)
    void* eta;           // per element [H][pitch][2] (storage precision)
    double* partial;     // per block maxima
    double* etamax;      // [batch]
    unsigned* cnt;
    double lam;
    double gms;
    const void* eld;      // K_rho element data or null
    long long eld_stride;
    const void* lamel;    // per-element lambda or null (constant)
    void* eldg;           // K_rho adjoint: 18 planes like eld (work)
    void* scratch;        // one [H][pitch] plane of the pair (work of the K_rho^T passes)
    const struct SmoothTaps* taps_rho;
    long long frame_off;  // the pair's frame offset (set per call)
    int pitch;
    double* vjp_w;        // adaptation-pass VJP work: dL/deta per element ([H][pitch][2] regions, FP64)
    double* vjp_buf;      // 26 planes of frame_elems doubles (13 per triangle family)
    double* vjp_part;     // block partials of the max(eta) term
    unsigned long long* vjp_argmax;
    int fp64;
};
cudaError_t launch_indicator(const AdaptBufs& A, int pair, int H, int W, cudaStream_t st);

// two-level preconditioner: A_0 blocks and dense scatter, symmetrisation of
// cuSOLVER's inverse, and one application z += R_0^T A_0^{-1} R_0 r (with the
// CG scalars finished unless apply_only); only_pair >= 0 restricts it to one pair
cudaError_t launch_coarse_assemble(const SolveBufs& B, cudaStream_t st);
cudaError_t launch_symmetrize(void* A, int fp64, int n, cudaStream_t st);
cudaError_t launch_coarse_apply(const SolveBufs& B, int first, int apply_only, int use_cond,
                                cudaGraphConditionalHandle cond, int only_pair, cudaStream_t st);
cudaError_t launch_coarse_factor(const SolveBufs& B, int pair, int n0, int nx, long long moff, cudaStream_t st);
cudaError_t coarse_configure(int fp64, int max_n0, int max_nx);

// K_sigma pre-smoothing: sampled Gaussian taps w_j of offsets j - r, j = 0..2r,
// and the prefix sums cw[i] = w_0 + ... + w_{i-1}
constexpr int OF_SMOOTH_RMAX = 48;
struct SmoothTaps {
    int r;
    double w[2 * OF_SMOOTH_RMAX + 1];
    double cw[2 * OF_SMOOTH_RMAX + 2];
};
// f ([H][pitch], type T_F32/T_F64) <- S f (or S^T f with transpose); scratch
// holds H x pitch values of the same type
cudaError_t launch_smooth(void* f, void* scratch, int type, int W, int H, long long pitch, const SmoothTaps& T,
                          bool transpose, cudaStream_t st);
// K_rho element data of one pair: eld (+ frame_off) gets 18 planes at stride
// `stride` (t * 9 + k: A_rho entries 00, 01, 02, 11, 12, 22, then F), each
// smoothed by T over the (W-1) x (H-1) lattice; scratch: H x pitch values
cudaError_t launch_element_data(const void* f1, const void* f2, int type, int W, int H, long long pitch, double gms,
                                void* eld, long long stride, void* scratch, const SmoothTaps& T, cudaStream_t st);
// the update rule of Section 2.3 on alpha, or on `field` (the per-element
// lambda) when it is not null
cudaError_t launch_alpha_update(const AdaptBufs& A, int pair, int H, int W, double kappa, double eta_thr,
                                double alpha_th, cudaStream_t st, void* field = nullptr);
// VJP of one adaptation pass (indicator at the stored solution, then the
// alpha update) for dL/dalpha_new = v (dense [H-1][W-1][2]): da = dL/dalpha
// through the pass, dU = dL/dU ([3][H][W]), df2 / df1 ([H][W], may be null)
cudaError_t launch_adapt_vjp(const AdaptBufs& A, int pair, int H, int W, double kappa, double eta_thr,
                             double alpha_th, const void* v, void* da, void* dU, void* df2, void* df1, int out_type,
                             cudaStream_t st);
// adjoint gradients for one pair: u = solution, lam = adjoint state (FP64 planes)
cudaError_t launch_adjoint_grad(const AdaptBufs& A, int pair, int H, int W, const double* lamv, void* dalpha,
                                void* df2, void* df1, int out_type, cudaStream_t st);

}  // namespace ofl
