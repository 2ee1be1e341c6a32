// Kernel instantiations and launchers of the solve path.
#include <functional>
#include <type_traits>

#include "of_apply.cuh"
#include "of_launch.h"
#include "of_schwarz.cuh"
#include "of_schwarz_h2.cuh"

namespace ofl {

using namespace ofk;

static constexpr int APPLY_NW = 4;    // warps per apply block (124 output columns)

// ------------------------------------------------------------ copy2d --
template <typename S, typename D>
__global__ void k_copy2d(const S* __restrict__ src, long long sp, D* __restrict__ dst, long long dp, long long rows,
                         long long cols) {
    const long long n = rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / cols, c = i - r * cols;
        if constexpr (std::is_same<S, double>::value && std::is_same<D, float>::value)
            dst[r * dp + c] = f32_from_double(src[r * sp + c]);  // off the FP64 pipe
        else
            dst[r * dp + c] = (D)src[r * sp + c];
    }
}
template <typename D>
__global__ void k_fill2d(D* dst, long long dp, long long rows, long long cols, D v) {
    const long long n = rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / cols, c = i - r * cols;
        dst[r * dp + c] = v;
    }
}

static unsigned grid_for(long long n, int nt) {
    long long g = (n + nt - 1) / nt;
    if (g > 152LL * 64) g = 152LL * 64;
    if (g < 1) g = 1;
    return (unsigned)g;
}

cudaError_t copy2d(const void* src, int stype, long long spitch, void* dst, int dtype, long long dpitch,
                   long long rows, long long cols, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const unsigned g = grid_for(rows * cols, 256);
    if (stype == T_F32 && dtype == T_F32)
        k_copy2d<float, float><<<g, 256, 0, st>>>((const float*)src, spitch, (float*)dst, dpitch, rows, cols);
    else if (stype == T_F32 && dtype == T_F64)
        k_copy2d<float, double><<<g, 256, 0, st>>>((const float*)src, spitch, (double*)dst, dpitch, rows, cols);
    else if (stype == T_F64 && dtype == T_F32)
        k_copy2d<double, float><<<g, 256, 0, st>>>((const double*)src, spitch, (float*)dst, dpitch, rows, cols);
    else
        k_copy2d<double, double><<<g, 256, 0, st>>>((const double*)src, spitch, (double*)dst, dpitch, rows, cols);
    return cudaGetLastError();
}

cudaError_t fill2d(void* dst, int dtype, long long dpitch, long long rows, long long cols, double v, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const unsigned g = grid_for(rows * cols, 256);
    if (dtype == T_F32) k_fill2d<float><<<g, 256, 0, st>>>((float*)dst, dpitch, rows, cols, (float)v);
    else k_fill2d<double><<<g, 256, 0, st>>>((double*)dst, dpitch, rows, cols, v);
    return cudaGetLastError();
}

// ------------------------------------------------------------- solve --
template <typename R, typename C, typename RI>
static ApplyParams<R, C, RI> base_params(const SolveBufs& B) {
    ApplyParams<R, C, RI> P;
    memset(&P, 0, sizeof(P));
    P.pairs = B.pairs;
    P.blocks = B.blocks;
    P.sc_in = B.sc;
    P.sc = B.sc;
    P.partial = B.partA;
    P.counter = B.cntA;
    P.gcounter = B.cntA + B.npairs;
    P.f1 = (const C*)B.f1;
    P.f2 = (const C*)B.f2;
    P.alpha = (const C*)B.alpha;
    P.lam = (R)B.lam;
    P.gms = (R)B.gms;
    P.eld = (const C*)B.eld;
    P.lamel = (const C*)B.lamel;
    P.eld_stride = B.eld_stride;
    P.rows_per_block = B.rows_per_block;
    P.err = B.err;
    return P;
}

template <typename C, typename RI>
static cudaError_t residual_t(const SolveBufs& B, const double* xin, double* xout, const double* rhs_vec, int first,
                              double rtol, double inner_rtol, double pass_frac, int max_inner, cudaStream_t st) {
    auto P = base_params<double, C, RI>(B);
    P.in = xin;
    P.p_buf0 = (RI*)B.p0;
    P.p_buf1 = (RI*)B.p1;
    P.dcorr = (RI*)B.d;
    P.out = xout;
    P.rout = (RI*)B.r;
    P.rhs_vec = rhs_vec;
    P.first = first;
    P.rtol = rtol;
    P.inner_rtol = inner_rtol;
    P.pass_frac = pass_frac;
    P.max_inner = max_inner;
    // the FP32 path forms A x and b in double-float: FP64-grade residual on the FP32 pipe
    using T = typename std::conditional<sizeof(C) == 4, DF, double>::type;
    if (B.eld) {
        if (xin) k_apply<double, C, RI, MODE_RES, false, APPLY_NW, T, true><<<B.nblk, APPLY_NW * 32, 0, st>>>(P);
        else k_apply<double, C, RI, MODE_RESB, false, APPLY_NW, T, true><<<B.nblk, APPLY_NW * 32, 0, st>>>(P);
    } else if (B.lamel) {
        if (xin) k_apply<double, C, RI, MODE_RES, false, APPLY_NW, T><<<B.nblk, APPLY_NW * 32, 0, st>>>(P);
        else k_apply<double, C, RI, MODE_RESB, false, APPLY_NW, T><<<B.nblk, APPLY_NW * 32, 0, st>>>(P);
    } else if (xin) {
        k_apply<double, C, RI, MODE_RES, false, APPLY_NW, T, false, false><<<B.nblk, APPLY_NW * 32, 0, st>>>(P);
    } else {
        // cold start (x = 0): r = b only seeds the first inner solve, whose
        // result the next residual (double-float) corrects, so the FP32 path
        // forms it in FP32 arithmetic (and ||b|| to FP32 accuracy)
        using TB = typename std::conditional<sizeof(C) == 4, float, double>::type;
        k_apply<double, C, RI, MODE_RESB, false, APPLY_NW, TB, false, false><<<B.nblk, APPLY_NW * 32, 0, st>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_residual(const SolveBufs& B, const double* xin, double* xout, const double* rhs_vec, int first,
                            double rtol, double inner_rtol, double pass_frac, int max_inner, cudaStream_t st) {
    if (B.fp64)
        return residual_t<double, double>(B, xin, xout, rhs_vec, first, rtol, inner_rtol, pass_frac, max_inner, st);
    return residual_t<float, float>(B, xin, xout, rhs_vec, first, rtol, inner_rtol, pass_frac, max_inner, st);
}

// One pair on the FP32 path with FP16 sweeps, one level and the four-column
// apply: the apply sums p.q as fixed-point integers (PairScalars::pq_fix),
// and every CTA of the Schwarz kernel that follows forms a = r.z / p.q.
static bool pq_fixed_point(const SolveBufs& B) {
    return B.h2 && !B.fp64 && B.npairs == 1 && !B.coarse.on && !B.eld && !B.lamel;
}

static SchwarzParams schwarz_params(const SolveBufs& B) {
    SchwarzParams S;
    memset(&S, 0, sizeof(S));
    S.pairs = B.pairs;
    S.tiles = B.tiles;
    S.ntiles = B.ntiles;
    S.npairs = B.npairs;
    S.tmaps = B.tmaps;
    S.ntab = B.ntab;
    S.sc = B.sc;
    S.partial = B.partS;
    S.counter = B.cntS;
    S.err = B.err;
    S.r = B.r;
    S.z = B.z;
    S.lam = B.lam;
    S.omega = B.omega;
    S.Tx = B.Tx;
    S.Ty = B.Ty;
    S.ov = B.ov;
    S.sweeps = B.sweeps;
    S.nstage = B.sch_nstage;
    S.spin_limit = B.spin_limit;
    S.use_cond = B.use_cond;
    S.tx_extra = B.tx_extra;
    S.cond = B.cond;
    S.pq_fixed = pq_fixed_point(B) ? 1 : 0;
    return S;
}

size_t schwarz_smem_bytes(int fp64, int Tx, int Ty, int ov, int nstage) {
    return fp64 ? sch_smem_bytes<double>(Tx, Ty, ov, nstage) : sch_smem_bytes<float>(Tx, Ty, ov, nstage);
}

// Tile shapes compiled with a compile-time geometry (the tuned ones);
// every other shape uses the runtime-geometry instantiation.
template <typename R, int NPT, typename F>
static cudaError_t with_schwarz(int tx, int ty, int ov, F f) {
    if (NPT == 2 && tx == 32 && ty == 32 && ov == 0) return f(k_schwarz<R, NPT, 32, 32, 0>);
    if (NPT == 2 && tx == 48 && ty == 48 && ov == 0) return f(k_schwarz<R, NPT, 48, 48, 0>);
    return f(k_schwarz<R, NPT, 0, 0, 0>);
}

// FP16 paired sweeps: the tuned shape with a compile-time geometry
template <typename F>
static cudaError_t with_schwarz_h2(int tx, int ty, int ov, F f) {
    if (tx == 48 && ty == 48 && ov == 0) return f(k_schwarz_h2<48, 48, 0>);
    return f(k_schwarz_h2<0, 0, 0>);
}

size_t schwarz_h2_smem_bytes(int Tx, int Ty, int ov, int nstage) { return h2_smem_bytes(Tx, Ty, ov, nstage); }

cudaError_t schwarz_h2_configure(int tx, int ty, int ov, size_t smem) {
    return with_schwarz_h2(tx, ty, ov, [&](auto kern) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
}

int schwarz_h2_max_grid(int tx, int ty, int ov, int threads, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    with_schwarz_h2(tx, ty, ov, [&](auto kern) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
    });
    if (per < 1) per = 1;
    return per * (sms > 0 ? sms : 1);
}

// Lane l of every warp takes a node whose z word lies in bank l (the sweeps'
// accesses), and within each warp the owned nodes are chosen so that their
// words of the dense Tx-wide r, q and z-out tiles also lie in distinct banks
// (the setup's and the emission's accesses): per colour, the nodes are the
// edges of a bipartite graph between z banks and tile banks, and each warp
// takes one matching of it (augmenting paths; the graph is regular for the
// tuned shapes, so every warp's matching is perfect; a node that cannot be
// matched is placed anyway, at the cost of a conflict).  Nodes of the overlap
// (not owned) touch no tile and match freely.
static void h2_assign_warps(const std::vector<std::vector<uint32_t>>& bucket, int Tx, int ov, int ns,
                            std::vector<std::vector<uint32_t>>& slots) {
    auto tile_bank = [&](uint32_t e) -> int {
        const int li = (int)(e & 0xffffu) - ov, lj = (int)(e >> 16) - ov;
        if (li < 0 || li >= Tx || lj < 0) return -1;  // not owned (lanes beyond the owned rows are checked in the kernel)
        return (int)(((long long)lj * Tx + li) % 32);
    };
    std::vector<std::vector<uint32_t>> left = bucket;  // remaining nodes per z bank
    slots.assign(ns, std::vector<uint32_t>(32, 0xffffffffu));
    for (int k = 0; k < ns; ++k) {
        // right vertices: 32 tile banks; owner[r] = the z bank matched to tile bank r, pick[b] = node index
        int owner[32], pick[32];
        for (int r = 0; r < 32; ++r) owner[r] = -1;
        for (int b = 0; b < 32; ++b) pick[b] = -1;
        for (int b = 0; b < 32; ++b) {
            if (left[b].empty()) continue;
            // a node of the overlap needs no tile bank
            for (size_t q = 0; q < left[b].size() && pick[b] < 0; ++q)
                if (tile_bank(left[b][q]) < 0) pick[b] = (int)q;
            if (pick[b] >= 0) continue;
            bool seen[32];
            std::function<bool(int)> augment = [&](int bb) -> bool {
                for (size_t q = 0; q < left[bb].size(); ++q) {
                    const int r = tile_bank(left[bb][q]);
                    if (r < 0 || seen[r]) continue;
                    seen[r] = true;
                    if (owner[r] < 0 || augment(owner[r])) {
                        owner[r] = bb;
                        pick[bb] = (int)q;
                        return true;
                    }
                }
                return false;
            };
            for (int r = 0; r < 32; ++r) seen[r] = false;
            if (!augment(b)) pick[b] = 0;  // unmatched: any node (a bank conflict)
        }
        for (int b = 0; b < 32; ++b) {
            if (pick[b] < 0) continue;
            slots[k][b] = left[b][pick[b]];
            left[b].erase(left[b].begin() + pick[b]);
        }
    }
    // anything left (never for the tuned shapes) goes to the first free lane slots of its z bank
    for (int b = 0; b < 32; ++b)
        for (uint32_t e : left[b])
            for (int k = 0; k < ns; ++k)
                if (slots[k][b] == 0xffffffffu) {
                    slots[k][b] = e;
                    break;
                }
}

bool schwarz_h2_node_table(int Tx, int Ty, int ov, std::vector<uint32_t>& tab, int& threads) {
    if (!h2_shape_ok(Ty, ov)) return false;
    const int Ex = Tx + 2 * ov, HP = h2_hp(Ty, ov), RW = sch_rw(Tx, ov), cpad = sch_cpad(ov);
    std::vector<std::vector<uint32_t>> slots[3];
    int maxslots = 0;
    for (int c = 0; c < 3; ++c) {
        std::vector<std::vector<uint32_t>> bucket(32);
        for (int j = 0; j < HP; ++j)
            for (int i = 0; i < Ex; ++i)
                if ((i + j) % 3 == c) bucket[((j + 1) * RW + (i + cpad - ov)) % 32].push_back((uint32_t)i | ((uint32_t)j << 16));
        size_t ns = 0;
        for (auto& b : bucket) ns = std::max(ns, b.size());
        h2_assign_warps(bucket, Tx, ov, (int)ns, slots[c]);
        maxslots = std::max(maxslots, (int)slots[c].size());
    }
    if (maxslots < 1 || maxslots > 12) return false;  // one pair per thread and colour, at most 384 threads
    threads = 32 * maxslots;
    tab.assign((size_t)3 * threads, 0xffffffffu);
    for (int c = 0; c < 3; ++c)
        for (size_t s = 0; s < slots[c].size(); ++s)
            for (int l = 0; l < 32; ++l) tab[(size_t)c * threads + s * 32 + l] = slots[c][s][l];
    return true;
}

template <typename F>
static cudaError_t with_schwarz_all(int fp64, int npt, int tx, int ty, int ov, F f) {
    if (fp64) return npt == 1 ? with_schwarz<double, 1>(tx, ty, ov, f) : with_schwarz<double, 2>(tx, ty, ov, f);
    return npt == 1 ? with_schwarz<float, 1>(tx, ty, ov, f) : with_schwarz<float, 2>(tx, ty, ov, f);
}

cudaError_t schwarz_configure(int fp64, int npt, int tx, int ty, int ov, size_t smem) {
    return with_schwarz_all(fp64, npt, tx, ty, ov, [&](auto kern) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
}

int schwarz_max_grid(int fp64, int npt, int tx, int ty, int ov, int threads, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    with_schwarz_all(fp64, npt, tx, ty, ov, [&](auto kern) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
    });
    if (per < 1) per = 1;
    return per * (sms > 0 ? sms : 1);
}

template <typename R>
static cudaError_t cells_t(const SolveBufs& B, int pair, int W, int H, void* c0, void* c1, cudaStream_t st) {
    dim3 grid((W + 127) / 128, H);
    k_cells<R><<<grid, 128, 0, st>>>(B.pairs, pair, (R)B.gms, (const R*)B.f1, (const R*)B.f2, (const R*)B.alpha,
                                    (typename CellT<R>::type*)c0, (typename CellT<R>::type*)c1);
    return cudaGetLastError();
}

namespace {
using namespace ofk;
// Paired element records of one pair from the FP16 records of k_cells:
// row k of the paired plane holds image row y = k - R (R = ov + 1 rows above
// the image, so that no tile's box starts above the plane), lane by lane
// (rec(x, y), rec(x, y + HP)) (see RecH2), each half zero where its row lies
// outside the image.
__global__ void k_cells_h2(const PairDesc* pairs, int pair, int HP, int R, const uint2* __restrict__ c0a,
                           const uint2* __restrict__ c1a, uint4* __restrict__ p0a, uint4* __restrict__ p1a, int* err) {
    const PairDesc pd = pairs[pair];
    const int x = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (x >= pd.W) return;
    const int y = k - R;
    const long long o = pd.frame_off + (long long)y * pd.pitch + x;
    const long long plane = (long long)pd.H * pd.pitch, lo = (long long)y * pd.pitch + x;
    const bool has_a = y >= 0 && y < pd.H && OF_CHECK(err, lo, plane);
    const bool has_b = y + HP >= 0 && y + HP < pd.H && OF_CHECK(err, lo + (long long)HP * pd.pitch, plane);
    const long long ob = o + (long long)HP * pd.pitch;
    // record words: x = (h0, h1), y = (h2, w); pair the low and the high halves
    auto pack = [](uint2 a, uint2 b) {
        return make_uint4(__byte_perm(a.x, b.x, 0x5410), __byte_perm(a.x, b.x, 0x7632),
                          __byte_perm(a.y, b.y, 0x5410), __byte_perm(a.y, b.y, 0x7632));
    };
    const uint2 zero = make_uint2(0u, 0u);
    if (!OF_CHECK(err, (long long)k * pd.pitch + x, (long long)(pd.H + R) * pd.pitch)) return;
    const long long po = pd.pair_off + (long long)k * pd.pitch + x;
    p0a[po] = pack(has_a ? c0a[o] : zero, has_b ? c0a[ob] : zero);
    p1a[po] = pack(has_a ? c1a[o] : zero, has_b ? c1a[ob] : zero);
}
}  // namespace

cudaError_t launch_cells(const SolveBufs& B, int pair, int W, int H, void* c0, void* c1, cudaStream_t st) {
    cudaError_t e = B.fp64 ? cells_t<double>(B, pair, W, H, c0, c1, st) : cells_t<float>(B, pair, W, H, c0, c1, st);
    if (e != cudaSuccess || !B.h2) return e;
    dim3 grid((W + 127) / 128, H + B.ov + 1);
    k_cells_h2<<<grid, 128, 0, st>>>(B.pairs, pair, h2_hp(B.Ty, B.ov), B.ov + 1, (const uint2*)c0,
                                     (const uint2*)c1, (uint4*)B.cp0, (uint4*)B.cp1, B.err);
    return cudaGetLastError();
}

bool schwarz_node_table(int fp64, int Tx, int Ty, int ov, std::vector<uint32_t>& tab, int& threads, int& npt) {
    const int Ex = Tx + 2 * ov, Ey = Ty + 2 * ov, RW = sch_rw(Tx, ov), cpad = sch_cpad(ov);
    const int nbank = fp64 ? 16 : 32;  // 8-byte words: 16 banks of pairs
    std::vector<std::vector<uint32_t>> slots[3];  // [colour][slot] -> up to 32 nodes, distinct banks
    int maxslots = 0;
    for (int c = 0; c < 3; ++c) {
        std::vector<std::vector<uint32_t>> bucket(nbank);
        for (int j = 0; j < Ey; ++j)
            for (int i = 0; i < Ex; ++i)
                if ((i + j) % 3 == c)
                    bucket[((j + 1) * RW + (i + cpad - ov)) % nbank].push_back((uint32_t)i | ((uint32_t)j << 16));
        size_t ns = 0;
        for (auto& b : bucket) ns = std::max(ns, b.size());
        // with 16 banks of 8-byte words, a warp takes two nodes per bank pair (two wavefronts anyway)
        const int per = 32 / nbank;
        slots[c].assign((ns + per - 1) / per, std::vector<uint32_t>(32, 0xffffffffu));
        for (int b = 0; b < nbank; ++b)
            for (size_t k = 0; k < bucket[b].size(); ++k) slots[c][k / per][b + nbank * (k % per)] = bucket[b][k];
        maxslots = std::max(maxslots, (int)slots[c].size());
    }
    // two nodes per thread and colour (independent updates in flight), as
    // many warps as that needs, at most the CTA cap
    int nwarps = (maxslots + 1) / 2;
    nwarps = std::min(std::max(nwarps, 1), sch_max_threads(fp64 != 0) / 32);
    npt = (maxslots + nwarps - 1) / nwarps;
    if (npt > 2) return false;
    threads = 32 * nwarps;
    tab.assign((size_t)3 * npt * threads, 0xffffffffu);
    for (int c = 0; c < 3; ++c)
        for (size_t s = 0; s < slots[c].size(); ++s) {
            const int k = (int)s / nwarps, w = (int)s % nwarps;
            for (int l = 0; l < 32; ++l) tab[((size_t)c * npt + k) * threads + w * 32 + l] = slots[c][s][l];
        }
    return true;
}

static cudaError_t schwarz_launch(const SolveBufs& B, const SchwarzParams& S, int ntiles, cudaStream_t st) {
    const int nt = B.sch_threads;
    const int grid = ntiles < B.sch_grid ? ntiles : B.sch_grid;
    if (grid <= 0) return cudaSuccess;
    SchwarzParams S2 = S;
    S2.ntiles = ntiles;
    if (B.h2) {
        const size_t smem = h2_smem_bytes(B.Tx, B.Ty, B.ov, B.sch_nstage);
        return with_schwarz_h2(B.Tx, B.Ty, B.ov, [&](auto kern) {
            kern<<<grid, nt, smem, st>>>(S2);
            return cudaGetLastError();
        });
    }
    const size_t smem = schwarz_smem_bytes(B.fp64, B.Tx, B.Ty, B.ov, B.sch_nstage);
    return with_schwarz_all(B.fp64, B.sch_npt, B.Tx, B.Ty, B.ov, [&](auto kern) {
        kern<<<grid, nt, smem, st>>>(S2);
        return cudaGetLastError();
    });
}

// Schwarz sweeps, then (two-level) the coarse correction, which finishes the
// CG scalars and, inside the loop graph, sets its condition
static cudaError_t precond(const SolveBufs& B, SchwarzParams S, int ntiles, int only_pair, cudaStream_t st) {
    if (!B.coarse.on) return schwarz_launch(B, S, ntiles, st);
    const int use_cond = S.use_cond;
    S.defer = 1;
    S.use_cond = 0;
    cudaError_t e = schwarz_launch(B, S, ntiles, st);
    if (e != cudaSuccess) return e;
    return launch_coarse_apply(B, S.first, S.apply_only, use_cond, B.cond, only_pair, st);
}

cudaError_t launch_precond_first(const SolveBufs& B, cudaStream_t st) {
    SchwarzParams S = schwarz_params(B);
    S.first = 1;
    return precond(B, S, B.ntiles, -1, st);
}

template <typename R>
static cudaError_t pcg_apply_t(const SolveBufs& B, cudaStream_t st) {
    auto P = base_params<R, R, R>(B);
    P.in = (const R*)B.z;
    P.p_buf0 = (R*)B.p0;
    P.p_buf1 = (R*)B.p1;
    P.dcorr = (R*)B.d;
    P.out = (R*)B.q;
    P.pq_fixed = pq_fixed_point(B) ? 1 : 0;
    if (B.eld) k_apply<R, R, R, MODE_PCG, false, APPLY_NW, R, true><<<B.nblk, APPLY_NW * 32, 0, st>>>(P);
    else if (B.lamel) k_apply<R, R, R, MODE_PCG, false, APPLY_NW><<<B.nblk, APPLY_NW * 32, 0, st>>>(P);  // per-element lambda
    else if constexpr (sizeof(R) == 4) k_apply4<MODE_PCG><<<B.nblk, 32, apply4_smem_bytes(), st>>>(P);  // FP32: four columns per lane
    else k_apply<R, R, R, MODE_PCG, false, APPLY_NW, R, false, false><<<B.nblk, APPLY_NW * 32, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_pcg_apply(const SolveBufs& B, cudaStream_t st) {
    return B.fp64 ? pcg_apply_t<double>(B, st) : pcg_apply_t<float>(B, st);
}

cudaError_t launch_pcg_precond(const SolveBufs& B, cudaStream_t st) {
    SchwarzParams S = schwarz_params(B);
    return precond(B, S, B.ntiles, -1, st);
}

template <typename R>
static cudaError_t apply_t(const SolveBufs& B, int blk0, int nblk, const void* p, void* q, void* b, cudaStream_t st) {
    auto P = base_params<R, R, R>(B);
    P.blocks = B.blocks + blk0;
    P.in = (const R*)p;
    P.out = (R*)q;
    P.bout = (R*)b;
    if (B.eld) {
        if (b) k_apply<R, R, R, MODE_APPLY, true, APPLY_NW, R, true><<<nblk, APPLY_NW * 32, 0, st>>>(P);
        else k_apply<R, R, R, MODE_APPLY, false, APPLY_NW, R, true><<<nblk, APPLY_NW * 32, 0, st>>>(P);
    } else if (b) k_apply<R, R, R, MODE_APPLY, true, APPLY_NW><<<nblk, APPLY_NW * 32, 0, st>>>(P);
    else if (B.lamel) k_apply<R, R, R, MODE_APPLY, false, APPLY_NW><<<nblk, APPLY_NW * 32, 0, st>>>(P);
    else if constexpr (sizeof(R) == 4) k_apply4<MODE_APPLY><<<nblk, 32, apply4_smem_bytes(), st>>>(P);
    else k_apply<R, R, R, MODE_APPLY, false, APPLY_NW, R, false, false><<<nblk, APPLY_NW * 32, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_apply(const SolveBufs& B, int pair, int blk0, int nblk, const void* p, void* q, void* b,
                         cudaStream_t st) {
    (void)pair;
    return B.fp64 ? apply_t<double>(B, blk0, nblk, p, q, b, st) : apply_t<float>(B, blk0, nblk, p, q, b, st);
}

cudaError_t launch_precond_only(const SolveBufs& B, int pair, int tile0, int ntiles, cudaStream_t st) {
    SchwarzParams S = schwarz_params(B);
    S.tiles = B.tiles + tile0;
    S.apply_only = 1;
    S.first = 1;
    return precond(B, S, ntiles, pair, st);
}

}  // namespace ofl
