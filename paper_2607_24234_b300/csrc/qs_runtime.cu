// qs_runtime.cu -- host runtime and C ABI of libqs.so (see include/qs.h).
//
// Host side (FP64): validation, the coefficient tables of the sweep
// (cos/sin of dxi and dxi/2, kappa = 1/(1+k^2), (q/m)/gamma, (q/m)/gamma^3,
// dt n_bs0(xi_j)), the transverse k set, the LPT-ordered work list, launch
// selection, the autotuner and CUDA-graph capture.  Device side: the kernels
// of qs_kernels.cuh, all enqueued on the context's stream.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "qs.h"
#include "qs_nvtx.h"
#include "qs_kernels.cuh"
#include "qs_problem.h"
#include "qs_resident.cuh"

using qsk::InstDev;
using qsk::SweepArgs;

namespace {

thread_local std::string g_init_err;

// Every context buffer carries a guard of CANARY_BYTES after its payload
// (at the payload size rounded up to 16 bytes), filled with CANARY_BYTE when
// it is allocated; qs_sync and host-pointer qs_diag check the guards, so a
// stray write past a buffer's end is reported (QS_ERR_BOUNDS) at the next
// synchronisation instead of corrupting a neighbour silently.
constexpr size_t CANARY_BYTES = 256;
constexpr unsigned char CANARY_BYTE = 0xA5;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    size_t canary = 0;   // offset of the guard
};

}  // namespace

struct qs_ctx {
    // problem
    qs_params p0;
    std::vector<qs_params> pin;     // per instance (copies; host pointers not kept)
    int n_inst = 1, prec = 0, NS = 1, M = 0, Mp = 0;
    std::vector<double> kx, ky, k2;
    std::vector<int> mode_id, partner_id;
    std::vector<InstDev> inst;
    std::vector<double> dens;       // [inst][2]
    long long cells_total = 0, groups_total = 0;
    // device
    qs_allocator alloc{};
    bool has_alloc = false;
    cudaStream_t stream = nullptr;
    std::vector<DevBuf> bufs;
    void *diag_tmp = nullptr;           // staging of host-form qs_diag results (kept: a free would
    size_t diag_tmp_bytes = 0;          // synchronise the whole device), one of bufs
    void *st = nullptr, *th = nullptr;
    int *ex = nullptr;
    InstDev *inst_d = nullptr;
    int2 *items_d = nullptr;
    int n_items = 0;
    // Green's-function path (qs_green.inc)
    bool uniform = false;           // every instance: the same dt n_bs0 in every cell
    bool theta_zero = false;        // Theta == 0 everywhere (fresh noise or user seed)
    std::vector<int> g_class_of, g_rep, g_mem_off, g_mem_mode;
    void *g_st = nullptr, *g_out = nullptr;
    int *g_ex = nullptr, *g_oex = nullptr, *g_mem_off_d = nullptr, *g_mem_mode_d = nullptr;
    double *g_kap = nullptr, *g_kapk2 = nullptr, *g_kabs = nullptr;
    int2 *g_items = nullptr;
    int g_n_items = 0, g_cap = 0;
    int2 *res_items_d = nullptr;    // resident variant: one item per CTA's lines
    int n_res_items = 0;
    long long res_key = -1;
    struct ResGroup { int threads, first, count; };
    std::vector<ResGroup> res_groups;   // instances sharing one CTA size, one launch each
    double *kap_d = nullptr, *kapk2_d = nullptr, *kabs_d = nullptr, *held_d = nullptr;
    void *w_d = nullptr;
    double *shape_d = nullptr, *dens_d = nullptr;
    int *mode_id_d = nullptr, *partner_d = nullptr;
    int *ticket_d = nullptr, *err_d = nullptr;
    size_t state_bytes = 0, th_bytes = 0, ex_bytes = 0;
    // run state
    long long step = 0;
    bool seeded = false, poisoned = false;
    int rec_kinds = 0, rec_stride = 1;
    long long rec_g0 = 0;
    void *rec_buf = nullptr;
    size_t rec_bytes = 0;
    qs_launch launch{2, 4, 0, 8, 0, 8};
    CUtensorMap tmA{}, tmB{};
    int tm_rows = -1;            // box rows the tensor maps were encoded for
    int items_for_warps = -1, items_persistent = -1;
    int n_sm = 148;
    std::map<int, cudaGraphExec_t> graphs;
    long long n_launch = 0;
    long long spin_limit = 1LL << 24;
    int tx_extra = 0;
    int res_every = 16;             // resident variant's renormalisation interval (0: variant refused)
    long long dbg_rows_cut = 0;     // test hook: state rows the bounds checker is told are missing
    bool uw_fit = false;            // uniform profile in every instance (the resident kernel's UW form)
    bool dbg_no_uw = false;         // QS_RES_NO_UNIFORM=1: the resident sweep reads per-cell weights even for a
                                    // uniform profile (compares the two kernels)
    double growth = 0.0;            // largest per-step growth bound of the instances (e-folds)
    std::string err;
};

namespace {

qs_status fail(qs_ctx *c, qs_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_init_err = buf;
    return st;
}

#define CU(c, x)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (x);                                                             \
        if (e_ != cudaSuccess) return fail((c), QS_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
    } while (0)

qs_status dalloc(qs_ctx *c, size_t bytes, void **out) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    const size_t guard = (bytes + 15) & ~size_t(15);
    bytes = guard + CANARY_BYTES;
    if (c->has_alloc) {
        p = c->alloc.alloc(bytes, c->alloc.user);
        if (!p) return fail(c, QS_ERR_OOM, "allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, e == cudaErrorMemoryAllocation ? QS_ERR_OOM : QS_ERR_CUDA,
                        "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        }
    }
    c->bufs.push_back({p, bytes, guard});
    if (cudaMemsetAsync(static_cast<char *>(p) + guard, CANARY_BYTE, CANARY_BYTES, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, QS_ERR_CUDA, "canary fill failed");
    }
    *out = p;
    return QS_OK;
}

template <typename P>
qs_status dalloc_t(qs_ctx *c, size_t bytes, P **out) {
    void *v = nullptr;
    qs_status s = dalloc(c, bytes, &v);
    *out = static_cast<P *>(v);
    return s;
}

qs_status upload(qs_ctx *c, void *dst, const void *src, size_t bytes) {
    CU(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    return QS_OK;
}

bool profile_shape(const qs_params &p, std::vector<double> &out) { return qsp::profile_shape(p, out); }

qs_status validate(const qs_params &p, int idx) {
    char msg[256];
    qs_status st = qsp::validate(p, idx, msg, sizeof msg);
    return st ? fail(nullptr, st, "%s", msg) : QS_OK;
}

// Transverse wavenumbers of the active modes (row-major over the grid).
void build_modes(qs_ctx *c, const qs_params &p) {
    qsp::ModeList m;
    qsp::build_modes(p, m);
    c->kx = std::move(m.kx); c->ky = std::move(m.ky); c->k2 = std::move(m.k2);
    c->mode_id = std::move(m.mode_id); c->partner_id = std::move(m.partner_id);
}

bool same_kset(const qs_params &a, const qs_params &b) {
    if (a.geom != b.geom) return false;
    if (a.geom == QS_GEOM_KLIST) {
        if (a.n_k != b.n_k) return false;
        for (int i = 0; i < a.n_k; ++i)
            if (a.k_list[i] != b.k_list[i]) return false;
        return true;
    }
    return a.nkx == b.nkx && a.nky == b.nky && a.kmax == b.kmax && a.disc_mask == b.disc_mask;
}

int max_nxi(const qs_ctx *c) {
    int mx = 0;
    for (const auto &I : c->inst) mx = std::max(mx, I.n_xi);
    return mx;
}

// threads holding one line in the resident variant (whole warps)
int res_threads_per_line(int n_xi, int V) { return ((n_xi + V - 1) / V + 31) & ~31; }

// CTA size of the resident variant for lines needing tl threads, at most
// Tmax: a whole number of lines (so no thread idles beyond the warp rounding
// of a line)
int res_cta_threads(int tl, int Tmax) { return tl * std::max(1, Tmax / tl); }
// Theta in registers at the largest cells per thread (launch.scan_cells)
bool res_regs(int NS, int V, int scan_cells) {
    return scan_cells == QS_RES_THETA_REGS && ((NS == 1 && V == 32) || (NS == 2 && V == 16));
}

// exact CTA sizes exist for every variant but two species at 16 cells per
// thread (Theta in shared memory, CTA of 128 | 256 | 512 threads only)
bool res_exact_sizes(int NS, int V, bool regs) { return regs || !(NS == 2 && V == 16); }

// Resident variant: an item is (instance, first mode) for the lines one CTA
// holds.  Instances are grouped by CTA size (one launch per group), longest
// lines first within a group when persistent.
qs_status build_res_items(qs_ctx *c) {
    const int V = c->launch.prefetch, Tmax = 32 * c->launch.warps_per_cta, P = c->launch.persistent;
    const bool regs = res_regs(c->NS, V, c->launch.scan_cells);
    const long long key = ((long long)V << 32) | ((long long)regs << 20) | ((long long)Tmax << 1) | P;
    if (c->res_key == key && c->res_items_d) return QS_OK;
    std::vector<int> order(c->n_inst);
    for (int i = 0; i < c->n_inst; ++i) order[i] = i;
    std::map<int, std::vector<int>> by_t;   // CTA size -> instances
    for (int i : order) {
        const int tl = res_threads_per_line(c->inst[i].n_xi, V);
        if (tl > Tmax) return fail(c, QS_ERR_ARG, "resident: a line of instance %d needs more than %d threads", i, Tmax);
        by_t[res_exact_sizes(c->NS, V, regs) ? res_cta_threads(tl, Tmax) : Tmax].push_back(i);
    }
    std::vector<int2> items;
    c->res_groups.clear();
    for (auto &g : by_t) {
        std::vector<int> &inst = g.second;
        if (P)
            std::stable_sort(inst.begin(), inst.end(),
                             [&](int a, int b) { return c->inst[a].n_xi > c->inst[b].n_xi; });
        const int first = (int)items.size();
        for (int i : inst) {
            const int L = g.first / res_threads_per_line(c->inst[i].n_xi, V);
            for (int m = 0; m < c->M; m += L) items.push_back(make_int2(i, m));
        }
        c->res_groups.push_back({g.first, first, (int)items.size() - first});
    }
    if (!c->res_items_d) {
        qs_status s = dalloc_t(c, (size_t)c->n_inst * c->M * sizeof(int2), &c->res_items_d);
        if (s) return s;
    }
    qs_status s = upload(c, c->res_items_d, items.data(), items.size() * sizeof(int2));
    if (s) return s;
    CU(c, cudaStreamSynchronize(c->stream));   // host vector dies at return
    c->n_res_items = (int)items.size();
    c->res_key = key;
    return QS_OK;
}

qs_status build_items(qs_ctx *c) {
    if (c->launch.variant == QS_VARIANT_RESIDENT) return build_res_items(c);
    // modes per work item: 32 x warps (thread per line), 32 (TMA), 32/S (scan)
    const int wpc = c->launch.variant == QS_VARIANT_TMA ? 1
                  : c->launch.variant == QS_VARIANT_SCAN ? -c->launch.prefetch
                  : c->launch.warps_per_cta;
    const int P = c->launch.persistent;
    if (c->items_for_warps == wpc && c->items_persistent == P && c->items_d) return QS_OK;
    const int per = wpc > 0 ? 32 * wpc : 32 / (-wpc);
    std::vector<int2> items;
    std::vector<int> order(c->n_inst);
    for (int i = 0; i < c->n_inst; ++i) order[i] = i;
    if (P)   // longest lines first (LPT)
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return c->inst[a].n_xi > c->inst[b].n_xi; });
    for (int i : order)
        for (int m = 0; m < c->M; m += per) items.push_back(make_int2(i, m));
    const size_t need = items.size() * sizeof(int2);
    // reuse the buffer when it is big enough (the maximum: one item per 32 modes)
    if (!c->items_d) {
        const size_t maxb = (size_t)c->n_inst * c->M * sizeof(int2);
        qs_status s = dalloc_t(c, maxb, &c->items_d);
        if (s) return s;
    }
    qs_status s = upload(c, c->items_d, items.data(), need);
    if (s) return s;
    CU(c, cudaStreamSynchronize(c->stream));   // host vector dies at return
    c->n_items = (int)items.size();
    c->items_for_warps = wpc;
    c->items_persistent = P;
    return QS_OK;
}

template <typename T, int NS, int U, bool REC>
cudaError_t launch_t(qs_ctx *c, const SweepArgs &a, dim3 grid, int threads) {
    qsk::k_sweep<T, NS, U, REC><<<grid, threads, 0, c->stream>>>(a);
    return cudaGetLastError();
}

template <typename T, int NS, bool REC>
cudaError_t launch_u(qs_ctx *c, const SweepArgs &a, dim3 grid, int threads, int U) {
    if constexpr (sizeof(T) == 4) {
        if (U >= 8) return launch_t<T, NS, 8, REC>(c, a, grid, threads);
        return launch_t<T, NS, 4, REC>(c, a, grid, threads);
    } else {
        if (U >= 4) return launch_t<T, NS, 4, REC>(c, a, grid, threads);
        return launch_t<T, NS, 2, REC>(c, a, grid, threads);
    }
}

// 2-D tensor maps over the state viewed as rows of Mp x 16 bytes:
// FP32: float elements, row = (cell, species), box = 32 modes x `rows` rows;
// FP64: double elements, one map for n_b and one for Theta.
qs_status ensure_tensor_maps(qs_ctx *c, int rows) {
    if (c->tm_rows == rows) return QS_OK;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(c, QS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const bool f32 = c->prec == QS_FP32_RENORM;
    const cuuint64_t dims[2] = {(cuuint64_t)c->Mp * (f32 ? 4 : 2), (cuuint64_t)c->cells_total * c->NS};
    const cuuint64_t strides[1] = {(cuuint64_t)c->Mp * 16};
    const cuuint32_t box[2] = {f32 ? 128u : 64u, (cuuint32_t)rows};
    const cuuint32_t es[2] = {1, 1};
    const CUtensorMapDataType dt = f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    CUresult r = encode(&c->tmA, dt, 2, c->st, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS && !f32)
        r = encode(&c->tmB, dt, 2, c->th, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, QS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    if (f32) c->tmB = c->tmA;
    c->tm_rows = rows;
    return QS_OK;
}

template <typename T, int NS, int C, int ST>
cudaError_t launch_tma_t(qs_ctx *c, const SweepArgs &a, dim3 grid) {
    qsk::k_sweep_tma<T, NS, C, ST><<<grid, 32, 0, c->stream>>>(a, c->tmA, c->tmB);
    return cudaGetLastError();
}

cudaError_t launch_tma(qs_ctx *c, const SweepArgs &a, dim3 grid, int C) {
    // ring depth chosen so that a CTA's buffers stay within 32 KiB of static shared memory
    if (c->prec == QS_FP32_RENORM) {
        if (c->NS == 1) return C >= 16 ? launch_tma_t<float, 1, 16, 3>(c, a, grid) : launch_tma_t<float, 1, 8, 4>(c, a, grid);
        return C >= 16 ? launch_tma_t<float, 2, 16, 2>(c, a, grid) : launch_tma_t<float, 2, 8, 4>(c, a, grid);
    }
    if (c->NS == 1) return C >= 8 ? launch_tma_t<double, 1, 8, 3>(c, a, grid) : launch_tma_t<double, 1, 4, 4>(c, a, grid);
    return C >= 8 ? launch_tma_t<double, 2, 8, 2>(c, a, grid) : launch_tma_t<double, 2, 4, 4>(c, a, grid);
}

template <int NS>
cudaError_t scan_ns(qs_ctx *c, const SweepArgs &a, dim3 grid, int threads, int S) {
    switch (S) {
    case 2: qsk::k_sweep_scan<NS, 2><<<grid, threads, 0, c->stream>>>(a); break;
    case 4: qsk::k_sweep_scan<NS, 4><<<grid, threads, 0, c->stream>>>(a); break;
    case 8: qsk::k_sweep_scan<NS, 8><<<grid, threads, 0, c->stream>>>(a); break;
    case 16: qsk::k_sweep_scan<NS, 16><<<grid, threads, 0, c->stream>>>(a); break;
    default: qsk::k_sweep_scan<NS, 32><<<grid, threads, 0, c->stream>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t scan_dispatch(qs_ctx *c, const SweepArgs &a, dim3 grid, int threads, int S) {
    return c->NS == 1 ? scan_ns<1>(c, a, grid, threads, S) : scan_ns<2>(c, a, grid, threads, S);
}

// One launch of the sweep kernel for n_steps steps starting at global step
// step0.  update = 0 runs the field pass only.  rec: record target (may be
// null).
SweepArgs sweep_args(qs_ctx *c, long long step0, int n_steps, int update, int rec_kinds,
                     double *rec, long long rec_g0, int rec_stride, long long rec_max_snap) {
    SweepArgs a{};
    a.st = c->st; a.th = c->th; a.ex = c->ex;
    a.inst = c->inst_d; a.items = c->items_d; a.n_items = c->n_items;
    a.kap = c->kap_d; a.kapk2 = c->kapk2_d; a.kabs = c->kabs_d; a.held = c->held_d;
    a.w = c->w_d;
    a.Mp = c->Mp; a.M = c->M; a.n_inst = c->n_inst;
    a.front = c->p0.front;
    a.step0 = step0; a.n_steps = n_steps; a.update = update;
    a.persistent = c->launch.persistent;
    a.rec_kinds = rec ? rec_kinds : 0;
    a.rec = rec; a.rec_g0 = rec_g0; a.rec_stride = rec_stride; a.rec_max_snap = rec_max_snap;
    a.cells_total = c->cells_total;
    const long long plane = c->cells_total * c->Mp;
    long long off = 0;
    a.rec_off_mag = off; if (rec_kinds & QS_REC_MAG) off += 5 * plane;
    a.rec_off_np = off;  if (rec_kinds & QS_REC_NP) off += 2 * plane;
    a.rec_off_mm = off;  if (rec_kinds & QS_REC_MODEMAX) off += 3LL * c->n_inst * c->Mp;
    a.rec_snap_doubles = off;
    a.ticket = c->ticket_d; a.err = c->err_d;
    a.scan_v = c->launch.scan_cells;
    a.spin_limit = c->spin_limit;
    a.tx_extra = c->tx_extra;
    a.res_every = c->res_every > 0 ? c->res_every : 1;
    a.rows_total = c->cells_total * c->NS - c->dbg_rows_cut;
    a.groups_total = c->groups_total;
    a.rec_cap = rec ? rec_max_snap * off : 0;
    return a;
}

template <int NS, int V, int TT, bool UW = false>
cudaError_t launch_res_t(qs_ctx *c, const SweepArgs &a, dim3 grid, int threads) {
    const size_t smem = qsk::res_smem_bytes(NS, V, TT, threads);
    // shared-memory opt-in (dynamic + static may pass 48 KiB), raised as larger CTAs appear
    static size_t opted = 0;
    if (smem > opted) {
        cudaError_t e = cudaFuncSetAttribute(qsk::k_sweep_res<NS, V, TT, UW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        opted = smem;
    }
    qsk::k_sweep_res<NS, V, TT, UW><<<grid, threads, smem, c->stream>>>(a);
    return cudaGetLastError();
}

// resident instantiations: Theta in registers (any CTA size) for 8 | 16 cells
// of one species and 8 of two; Theta in shared memory for 32 cells of one
// species (CTA of 64 | 128 | 256) and 16 of two (CTA of 128 | 256 | 512), or,
// with `regs`, in registers there too (255 registers, CTA of at most 256)
cudaError_t launch_res(qs_ctx *c, const SweepArgs &a, dim3 grid, int T, int V, bool regs) {
    if (regs && c->NS == 1 && V == 32) return T <= 256 ? launch_res_t<1, 32, 0>(c, a, grid, T) : cudaErrorInvalidValue;
    if (regs && c->NS == 2 && V == 16) return T <= 256 ? launch_res_t<2, 16, 0>(c, a, grid, T) : cudaErrorInvalidValue;
    if (c->NS == 1) {
        // uniform profiles: the cell weight in a register
        if (V == 32 && c->uw_fit && !c->dbg_no_uw) switch (T) {
            case 64: return launch_res_t<1, 32, 64, true>(c, a, grid, T);
            case 96: return launch_res_t<1, 32, 96, true>(c, a, grid, T);
            case 128: return launch_res_t<1, 32, 128, true>(c, a, grid, T);
            case 160: return launch_res_t<1, 32, 160, true>(c, a, grid, T);
            case 192: return launch_res_t<1, 32, 192, true>(c, a, grid, T);
            case 224: return launch_res_t<1, 32, 224, true>(c, a, grid, T);
            case 256: return launch_res_t<1, 32, 256, true>(c, a, grid, T);
            default: return cudaErrorInvalidValue;
            }
        if (V == 32) switch (T) {   // every whole number of 64-thread lines up to 4, and 96 .. 224 for 96-thread lines
            case 64: return launch_res_t<1, 32, 64>(c, a, grid, T);
            case 96: return launch_res_t<1, 32, 96>(c, a, grid, T);
            case 128: return launch_res_t<1, 32, 128>(c, a, grid, T);
            case 160: return launch_res_t<1, 32, 160>(c, a, grid, T);
            case 192: return launch_res_t<1, 32, 192>(c, a, grid, T);
            case 224: return launch_res_t<1, 32, 224>(c, a, grid, T);
            case 256: return launch_res_t<1, 32, 256>(c, a, grid, T);
            default: return cudaErrorInvalidValue;   // no kernel for this CTA size
            }
        return V == 16 ? launch_res_t<1, 16, 0>(c, a, grid, T) : launch_res_t<1, 8, 0>(c, a, grid, T);
    }
    if (V == 16) return T == 128 ? launch_res_t<2, 16, 128>(c, a, grid, T)
                      : T == 256 ? launch_res_t<2, 16, 256>(c, a, grid, T)
                      : T == 512 ? launch_res_t<2, 16, 512>(c, a, grid, T)
                                 : cudaErrorInvalidValue;
    return launch_res_t<2, 8, 0>(c, a, grid, T);
}

bool res_shape_ok(int NS, int V, int w, bool regs = false) {
    if (regs) return res_regs(NS, V, QS_RES_THETA_REGS) && (w == 1 || w == 2 || w == 4 || w == 8);
    if (NS == 1 && V == 32) return w == 2 || w == 4 || w == 8;
    if (NS == 2 && V == 16) return w == 4 || w == 8 || w == 16;
    return (V == 8 || (V == 16 && NS == 1)) && (w == 1 || w == 2 || w == 4 || w == 8 || w == 16);
}

qs_status launch_sweep(qs_ctx *c, long long step0, int n_steps, int update, int rec_kinds,
                       double *rec, long long rec_g0, int rec_stride, long long rec_max_snap);

// Resident variant: updating steps without records run on chip; a step that
// records, and every field pass, runs the register kernel (same per-cell
// arithmetic) on its own work list.
qs_status launch_resident(qs_ctx *c, long long step0, int n_steps, int update, int rec_kinds,
                          double *rec, long long rec_g0, int rec_stride, long long rec_max_snap) {
    auto fallback = [&](long long s0, int n, int upd) {
        const qs_launch keep = c->launch;
        c->launch = qs_launch{1, 8, 0, 8, QS_VARIANT_REGISTERS, 8};
        qs_status r = launch_sweep(c, s0, n, upd, rec_kinds, rec, rec_g0, rec_stride, rec_max_snap);
        c->launch = keep;
        return r;
    };
    // the per-mode maxima are computed on chip; full field snapshots are not
    const bool mm_only = rec && rec_kinds == QS_REC_MODEMAX;
    if (!update && !mm_only) return fallback(step0, n_steps, 0);
    const bool recording = rec && rec_kinds && !mm_only;
    const long long end = step0 + n_steps;
    long long cur = step0;
    while (cur < end) {
        long long r = end;   // next step that records
        if (recording) {
            const long long d = cur - rec_g0;
            const long long cand = d <= 0 ? rec_g0 : rec_g0 + ((d + rec_stride - 1) / rec_stride) * rec_stride;
            if (cand < end && (cand - rec_g0) / rec_stride < rec_max_snap) r = cand;
        }
        if (r > cur) {
            qs_status s = build_res_items(c);
            if (s) return s;
            SweepArgs a = mm_only ? sweep_args(c, cur, (int)(r - cur), update, rec_kinds, rec, rec_g0, rec_stride,
                                               rec_max_snap)
                                  : sweep_args(c, cur, (int)(r - cur), 1, 0, nullptr, 0, 1, 0);
            for (const auto &grp : c->res_groups) {   // one launch per CTA size
                a.items = c->res_items_d + grp.first;
                a.n_items = grp.count;
                dim3 grid(grp.count);
                if (a.persistent) {
                    CU(c, cudaMemsetAsync(c->ticket_d, 0, sizeof(int), c->stream));
                    const long long g = (long long)c->launch.ctas_per_sm * c->n_sm;
                    grid = dim3((unsigned)std::max<long long>(1, std::min<long long>(g, grp.count)));
                }
                cudaError_t e = launch_res(c, a, grid, grp.threads, c->launch.prefetch,
                                           res_regs(c->NS, c->launch.prefetch, c->launch.scan_cells));
                if (e != cudaSuccess) return fail(c, QS_ERR_CUDA, "resident sweep launch: %s", cudaGetErrorString(e));
                ++c->n_launch;
            }
        }
        if (r < end) {
            qs_status s = fallback(r, 1, 1);
            if (s) return s;
        }
        cur = r + 1;
    }
    return QS_OK;
}

qs_status launch_sweep(qs_ctx *c, long long step0, int n_steps, int update, int rec_kinds,
                       double *rec, long long rec_g0, int rec_stride, long long rec_max_snap) {
    if (c->launch.variant == QS_VARIANT_RESIDENT)
        return launch_resident(c, step0, n_steps, update, rec_kinds, rec, rec_g0, rec_stride, rec_max_snap);
    qs_status s = build_items(c);
    if (s) return s;
    SweepArgs a = sweep_args(c, step0, n_steps, update, rec_kinds, rec, rec_g0, rec_stride, rec_max_snap);
    const bool use_tma = c->launch.variant == QS_VARIANT_TMA && update && !rec_kinds;
    const bool use_scan = c->launch.variant == QS_VARIANT_SCAN && update && !rec_kinds && c->prec == QS_FP64;
    if (c->launch.variant == QS_VARIANT_SCAN && !use_scan) {
        // field / record passes of a scan-configured context run the register
        // kernel (same per-cell arithmetic) with its own work list
        const qs_launch keep = c->launch;
        c->launch = qs_launch{1, c->prec == QS_FP32_RENORM ? 8 : 4, 0, 8, QS_VARIANT_REGISTERS, 8};
        qs_status r = launch_sweep(c, step0, n_steps, update, rec_kinds, rec, rec_g0, rec_stride, rec_max_snap);
        c->launch = keep;
        c->items_for_warps = -1000;   // force the scan work list to be rebuilt
        return r;
    }
    const int threads = 32 * (c->launch.variant == QS_VARIANT_TMA ? 1 : c->launch.warps_per_cta);
    dim3 grid(c->n_items);
    if (a.persistent) {
        CU(c, cudaMemsetAsync(c->ticket_d, 0, sizeof(int), c->stream));
        long long g = (long long)c->launch.ctas_per_sm * c->n_sm;
        grid = dim3((unsigned)std::max<long long>(1, std::min<long long>(g, c->n_items)));
    }
    const bool R = a.rec_kinds != 0;
    const int U = c->launch.prefetch;
    cudaError_t e;
    if (use_scan) {
        const int S = c->launch.prefetch;
        const int wpb = c->launch.warps_per_cta;
        a.persistent = 0;
        const dim3 g2((unsigned)((c->n_items + wpb - 1) / wpb));
        e = scan_dispatch(c, a, g2, 32 * wpb, S);
    } else if (use_tma) {
        const int C = c->launch.prefetch;
        const int rows = (c->prec == QS_FP32_RENORM ? (C >= 16 ? 16 : 8) : (C >= 8 ? 8 : 4)) * c->NS;
        qs_status ts = ensure_tensor_maps(c, rows);
        if (ts) return ts;
        e = launch_tma(c, a, grid, C);
    } else if (c->launch.variant == QS_VARIANT_TMA) {
        // record / field passes of a TMA-configured context: the register
        // kernel with the same per-cell arithmetic, one warp per CTA
        e = c->prec == QS_FP32_RENORM
                ? (c->NS == 1 ? (R ? launch_u<float, 1, true>(c, a, grid, threads, 8) : launch_u<float, 1, false>(c, a, grid, threads, 8))
                              : (R ? launch_u<float, 2, true>(c, a, grid, threads, 8) : launch_u<float, 2, false>(c, a, grid, threads, 8)))
                : (c->NS == 1 ? (R ? launch_u<double, 1, true>(c, a, grid, threads, 4) : launch_u<double, 1, false>(c, a, grid, threads, 4))
                              : (R ? launch_u<double, 2, true>(c, a, grid, threads, 4) : launch_u<double, 2, false>(c, a, grid, threads, 4)));
    } else if (c->prec == QS_FP32_RENORM) {
        if (c->NS == 1) e = R ? launch_u<float, 1, true>(c, a, grid, threads, U) : launch_u<float, 1, false>(c, a, grid, threads, U);
        else e = R ? launch_u<float, 2, true>(c, a, grid, threads, U) : launch_u<float, 2, false>(c, a, grid, threads, U);
    } else {
        if (c->NS == 1) e = R ? launch_u<double, 1, true>(c, a, grid, threads, U) : launch_u<double, 1, false>(c, a, grid, threads, U);
        else e = R ? launch_u<double, 2, true>(c, a, grid, threads, U) : launch_u<double, 2, false>(c, a, grid, threads, U);
    }
    if (e != cudaSuccess) return fail(c, QS_ERR_CUDA, "sweep launch: %s", cudaGetErrorString(e));
    ++c->n_launch;
    return QS_OK;
}

long long snapshot_doubles(const qs_ctx *c, int kinds) {
    const long long plane = c->cells_total * c->Mp;
    long long d = 0;
    if (kinds & QS_REC_MAG) d += 5 * plane;
    if (kinds & QS_REC_NP) d += 2 * plane;
    if (kinds & QS_REC_MODEMAX) d += 3LL * c->n_inst * c->Mp;
    return d;
}

// guard check: one CTA per buffer compares its CANARY_BYTES with the fill;
// a mismatch sets ERR_CANARY and keeps the buffer index + 1 in word 1
struct CanaryArgs {
    const uint4 *p[32];
    int n, first;
    int *err;
};
__global__ void k_canary(const CanaryArgs a) {
    const int b = blockIdx.x;
    if (b >= a.n) return;
    const uint4 v = a.p[b][threadIdx.x];
    const unsigned f = 0x01010101u * CANARY_BYTE;
    if (v.x != f || v.y != f || v.z != f || v.w != f) {
        atomicOr(a.err, qsk::ERR_CANARY);
        atomicCAS(a.err + 1, 0, a.first + b + 1);
    }
}

qs_status check_canaries(qs_ctx *c) {
    for (size_t b0 = 0; b0 < c->bufs.size(); b0 += 32) {
        CanaryArgs a{};
        a.n = (int)std::min<size_t>(32, c->bufs.size() - b0);
        a.first = (int)b0;
        a.err = c->err_d;
        for (int i = 0; i < a.n; ++i)
            a.p[i] = reinterpret_cast<const uint4 *>(static_cast<const char *>(c->bufs[b0 + i].p) + c->bufs[b0 + i].canary);
        k_canary<<<a.n, CANARY_BYTES / 16, 0, c->stream>>>(a);
        CU(c, cudaGetLastError());
    }
    return QS_OK;
}

qs_status check_ready(qs_ctx *c) {
    if (!c) return QS_ERR_ARG;
    if (c->poisoned) return fail(c, QS_ERR_STATE, "context poisoned by an earlier device error; reseed");
    if (!c->seeded) return fail(c, QS_ERR_STATE, "qs_seed has not been called");
    return QS_OK;
}

}  // namespace

extern "C" {

qs_status qs_init(const qs_params *p, int n_inst, const qs_params *per_inst,
                  const qs_allocator *alloc, void *stream, qs_ctx **out) {
    QS_RANGE("qs_init");
    if (!p || !out) return fail(nullptr, QS_ERR_ARG, "null params or out");
    *out = nullptr;
    if (n_inst < 1) return fail(nullptr, QS_ERR_ARG, "n_inst must be >= 1");
    qs_status st = validate(*p, -1);
    if (st) return st;
    for (int i = 0; per_inst && i < n_inst; ++i) {
        const qs_params &q = per_inst[i];
        if ((st = validate(q, i))) return st;
        if (q.prec != p->prec || q.model != p->model || q.front != p->front ||
            q.n_species != p->n_species || !same_kset(q, *p))
            return fail(nullptr, QS_ERR_ARG, "instance %d differs from the shared params in "
                        "prec/model/front/n_species/k set", i);
    }
    qs_ctx *c = new qs_ctx();
    c->p0 = *p;
    c->n_inst = n_inst;
    c->prec = p->prec;
    c->NS = p->n_species;
    c->stream = static_cast<cudaStream_t>(stream);
    if (alloc && alloc->alloc && alloc->free) { c->alloc = *alloc; c->has_alloc = true; }
    build_modes(c, *p);
    c->M = (int)c->k2.size();
    if (c->M < 1) { delete c; return fail(nullptr, QS_ERR_ARG, "no active mode (disc mask empty)"); }
    c->Mp = (c->M + 31) / 32 * 32;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) c->n_sm = v;
    } else {
        cudaGetLastError();
    }
    // per-instance tables
    std::vector<double> shape_all, w_all;
    c->inst.resize(n_inst);
    c->dens.assign(2 * (size_t)n_inst, 0.0);
    long long cell = 0, grp = 0;
    for (int i = 0; i < n_inst; ++i) {
        const qs_params &q = per_inst ? per_inst[i] : *p;
        std::vector<double> shp;
        if (!profile_shape(q, shp)) { delete c; return fail(nullptr, QS_ERR_ARG, "instance %d: profile", i); }
        InstDev &I = c->inst[i];
        I.n_xi = q.n_xi;
        I.n_grp = (q.n_xi + qsk::GRP - 1) / qsk::GRP;
        I.cell_off = cell;
        I.grp_off = grp;
        I.noise_inst = i;
        I.c = std::cos(q.dxi); I.s = std::sin(q.dxi);
        I.ch = std::cos(0.5 * q.dxi); I.sh = std::sin(0.5 * q.dxi);
        I.dt = q.dt; I.dxi = q.dxi;
        const double g = q.gamma_b;
        for (int s = 0; s < 2; ++s) {
            if (s < q.n_species) {
                const double qm = q.species[s].q / q.species[s].m;
                I.q[s] = q.species[s].q;
                I.qm_g[s] = qm / g;
                I.qm_g3[s] = q.model == QS_MODEL_REDUCED ? 0.0 : qm / (g * g * g);
                c->dens[2 * i + s] = q.species[s].density_ratio;
            } else {
                I.q[s] = 0.0; I.qm_g[s] = 0.0; I.qm_g3[s] = 0.0;
            }
        }
        bool uni = true;
        for (int j = 0; j < q.n_xi; ++j) {
            shape_all.push_back(shp[j]);
            for (int s = 0; s < c->NS; ++s) w_all.push_back(q.dt * q.species[s].density_ratio * shp[j]);
            uni = uni && shp[j] == shp[0];
        }
        for (int s = 0; s < 2; ++s)   // the cell weight of a uniform profile, as the FP32 path stores it
            I.wu[s] = s < c->NS ? (float)(q.dt * q.species[s].density_ratio * shp[0]) : 0.0f;
        c->uniform = (i == 0 || c->uniform) && uni;
        {
            double lc = 0.0;
            const double gb = qsp::growth_bound(q, shp, &lc);
            c->growth = std::max(c->growth, gb);
            const int ev = qsp::res_every_for(gb, lc, q.n_xi * q.dxi);
            c->res_every = i == 0 ? ev : std::min(c->res_every, ev);
        }
        cell += q.n_xi;
        grp += I.n_grp;
    }
    c->cells_total = cell;
    c->groups_total = grp;
    if (const char *v = getenv("QS_RES_NO_UNIFORM")) c->dbg_no_uw = v[0] == '1';
    c->uw_fit = c->uniform;
    c->pin.assign(n_inst, *p);
    for (int i = 0; per_inst && i < n_inst; ++i) c->pin[i] = per_inst[i];
    // per-mode tables (padding modes: k = 0, never stepped)
    std::vector<double> kap(c->Mp, 1.0), kapk2(c->Mp, 0.0), kabs(c->Mp, 0.0);
    std::vector<int> mid(c->Mp, 0), pid(c->Mp, 0);
    for (int m = 0; m < c->M; ++m) {
        kap[m] = 1.0 / (1.0 + c->k2[m]);
        kapk2[m] = c->k2[m] * kap[m];
        kabs[m] = std::sqrt(c->k2[m]);
        mid[m] = c->mode_id[m];
        pid[m] = c->partner_id[m];
    }
    // device buffers
    const size_t rows = (size_t)c->cells_total * c->NS;
    const size_t esz = c->prec == QS_FP32_RENORM ? sizeof(float4) : sizeof(double2);
    c->state_bytes = rows * c->Mp * esz;
    c->th_bytes = c->prec == QS_FP64 ? c->state_bytes : 0;
    c->ex_bytes = c->prec == QS_FP32_RENORM ? (size_t)c->groups_total * c->Mp * sizeof(int) : 0;
#define ALLOC(ptr, bytes) do { if ((st = dalloc_t(c, (bytes), &(ptr)))) { qs_free(c); g_init_err = "allocation failed"; return st; } } while (0)
    ALLOC(c->st, c->state_bytes);
    if (c->th_bytes) ALLOC(c->th, c->th_bytes);
    if (c->ex_bytes) ALLOC(c->ex, c->ex_bytes);
    ALLOC(c->inst_d, sizeof(InstDev) * n_inst);
    ALLOC(c->kap_d, sizeof(double) * c->Mp);
    ALLOC(c->kapk2_d, sizeof(double) * c->Mp);
    ALLOC(c->kabs_d, sizeof(double) * c->Mp);
    ALLOC(c->shape_d, sizeof(double) * c->cells_total);
    ALLOC(c->dens_d, sizeof(double) * 2 * n_inst);
    ALLOC(c->mode_id_d, sizeof(int) * c->Mp);
    ALLOC(c->partner_d, sizeof(int) * c->Mp);
    ALLOC(c->ticket_d, sizeof(int) * 4);
    ALLOC(c->err_d, sizeof(int) * 4);
    ALLOC(c->w_d, (c->prec == QS_FP32_RENORM ? sizeof(float) : sizeof(double)) * rows);
    if (p->front == QS_FRONT_HELD) ALLOC(c->held_d, sizeof(double) * 4 * (size_t)n_inst * c->Mp);
#undef ALLOC
    auto up = [&](void *d, const void *h, size_t b) -> qs_status {
        cudaError_t e = cudaMemcpy(d, h, b, cudaMemcpyHostToDevice);
        return e == cudaSuccess ? QS_OK : fail(c, QS_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    };
    std::vector<float> wf;
    if (c->prec == QS_FP32_RENORM) { wf.assign(w_all.begin(), w_all.end()); }
    if ((st = up(c->inst_d, c->inst.data(), sizeof(InstDev) * n_inst)) ||
        (st = up(c->kap_d, kap.data(), sizeof(double) * c->Mp)) ||
        (st = up(c->kapk2_d, kapk2.data(), sizeof(double) * c->Mp)) ||
        (st = up(c->kabs_d, kabs.data(), sizeof(double) * c->Mp)) ||
        (st = up(c->shape_d, shape_all.data(), sizeof(double) * c->cells_total)) ||
        (st = up(c->dens_d, c->dens.data(), sizeof(double) * 2 * n_inst)) ||
        (st = up(c->mode_id_d, mid.data(), sizeof(int) * c->Mp)) ||
        (st = up(c->partner_d, pid.data(), sizeof(int) * c->Mp)) ||
        (st = up(c->w_d, c->prec == QS_FP32_RENORM ? (const void *)wf.data() : (const void *)w_all.data(),
                 (c->prec == QS_FP32_RENORM ? sizeof(float) : sizeof(double)) * rows))) {
        g_init_err = c->err; qs_free(c); return st;
    }
    if (c->held_d) {
        std::vector<double> h(4 * (size_t)n_inst * c->Mp, 0.0);
        for (int i = 0; i < n_inst; ++i) {
            const double *src = (per_inst ? per_inst[i] : *p).held_front;
            for (int m = 0; m < c->M; ++m)
                for (int k = 0; k < 4; ++k) h[((size_t)i * c->Mp + m) * 4 + k] = src[4 * m + k];
        }
        if ((st = up(c->held_d, h.data(), h.size() * sizeof(double)))) { g_init_err = c->err; qs_free(c); return st; }
    }
    cudaError_t e1 = cudaMemsetAsync(c->st, 0, c->state_bytes, c->stream);
    cudaError_t e2 = c->th ? cudaMemsetAsync(c->th, 0, c->th_bytes, c->stream) : cudaSuccess;
    cudaError_t e3 = c->ex ? cudaMemsetAsync(c->ex, 0, c->ex_bytes, c->stream) : cudaSuccess;
    cudaError_t e4 = cudaMemsetAsync(c->err_d, 0, 4 * sizeof(int), c->stream);
    if (e1 || e2 || e3 || e4) { g_init_err = "memset failed"; qs_free(c); return QS_ERR_CUDA; }
    // default launch shape: the FP64 path keeps fewer cells in flight per thread
    // default launch shape (measured on B300 for the 3D beam workload): TMA
    // tiles of 8 (FP32) / 4 (FP64) cells x 32 modes, 4-deep ring; batched
    // contexts pull an LPT-ordered work list
    c->launch = qs_launch{1, c->prec == QS_FP32_RENORM ? 8 : 4, n_inst > 1 ? 1 : 0, 16, QS_VARIANT_TMA, 8};
    *out = c;
    return QS_OK;
}

qs_status qs_seed(qs_ctx *c, uint64_t seed, double amplitude, int kind, const void *user,
                  size_t user_bytes, int user_on_host) {
    QS_RANGE("qs_seed");
    if (!c) return QS_ERR_ARG;
    if (kind < 0 || kind > 3) return fail(c, QS_ERR_ARG, "seed kind %d", kind);
    if (kind == QS_SEED_STATE) {
        // checkpoint: header (8 int64) + state + theta + exponents
        const size_t need = 64 + c->state_bytes + c->th_bytes + c->ex_bytes;
        if (!user || user_bytes < need) return fail(c, QS_ERR_ARG, "checkpoint needs %zu bytes", need);
        int64_t hdr[8];
        cudaMemcpyKind k = user_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        if (user_on_host) memcpy(hdr, user, 64);
        else {
            CU(c, cudaMemcpyAsync(hdr, user, 64, cudaMemcpyDeviceToHost, c->stream));
            CU(c, cudaStreamSynchronize(c->stream));
        }
        if (hdr[0] != 0x51534350 || hdr[1] != c->prec || hdr[2] != c->NS || hdr[3] != c->Mp ||
            hdr[4] != c->cells_total)
            return fail(c, QS_ERR_ARG, "checkpoint does not match this context");
        const char *u = static_cast<const char *>(user) + 64;
        CU(c, cudaMemcpyAsync(c->st, u, c->state_bytes, k, c->stream));
        if (c->th_bytes) CU(c, cudaMemcpyAsync(c->th, u + c->state_bytes, c->th_bytes, k, c->stream));
        if (c->ex_bytes) CU(c, cudaMemcpyAsync(c->ex, u + c->state_bytes + c->th_bytes, c->ex_bytes, k, c->stream));
        if (user_on_host) CU(c, cudaStreamSynchronize(c->stream));
        c->step = hdr[5];
    } else {
        qsk::SeedArgs a{};
        a.st = c->st; a.th = c->th; a.ex = c->ex;
        a.inst = c->inst_d; a.shape = c->shape_d; a.dens = c->dens_d;
        a.mode_id = c->mode_id_d; a.partner_id = c->partner_d;
        a.Mp = c->Mp; a.M = c->M; a.NS = c->NS; a.n_inst = c->n_inst;
        a.kind = kind; a.seed = seed; a.amp = amplitude;
        a.total_groups = c->groups_total;
        void *tmp = nullptr;
        if (kind == QS_SEED_IMPULSE) {
            for (int i = 0; i < c->n_inst; ++i)
                if (!(c->pin[i].species[0].q != 0.0) || !(c->dens[2 * i] > 0.0))
                    return fail(c, QS_ERR_ARG, "impulse seed needs q_0 != 0 and n_b00 > 0");
        }
        if (kind == QS_SEED_USER) {
            const size_t need = (size_t)c->M * c->NS * c->cells_total * 16;
            if (!user || user_bytes < need) return fail(c, QS_ERR_ARG, "user seed needs %zu bytes", need);
            if (user_on_host) {
                qs_status s = dalloc(c, need, &tmp);
                if (s) return s;
                CU(c, cudaMemcpyAsync(tmp, user, need, cudaMemcpyHostToDevice, c->stream));
                a.user = static_cast<const double *>(tmp);
            } else {
                a.user = static_cast<const double *>(user);
            }
        }
        CU(c, cudaMemsetAsync(c->st, 0, c->state_bytes, c->stream));
        if (c->th) CU(c, cudaMemsetAsync(c->th, 0, c->th_bytes, c->stream));
        dim3 grid((c->Mp + 127) / 128, (unsigned)std::min<long long>(c->groups_total, 65535),
                  (unsigned)((c->groups_total + 65534) / 65535));
        if (c->prec == QS_FP32_RENORM) qsk::k_seed<float><<<grid, 128, 0, c->stream>>>(a);
        else qsk::k_seed<double><<<grid, 128, 0, c->stream>>>(a);
        CU(c, cudaGetLastError());
        if (tmp) {
            CU(c, cudaStreamSynchronize(c->stream));
            // release the staging buffer now
            for (size_t i = 0; i < c->bufs.size(); ++i)
                if (c->bufs[i].p == tmp) {
                    if (c->has_alloc) c->alloc.free(tmp, c->alloc.user); else cudaFree(tmp);
                    c->bufs.erase(c->bufs.begin() + i);
                    break;
                }
        }
        c->step = 0;
    }
    CU(c, cudaMemsetAsync(c->err_d, 0, 4 * sizeof(int), c->stream));
    c->seeded = true;
    c->theta_zero = kind == QS_SEED_NOISE || kind == QS_SEED_USER;   // these seeds leave Theta = 0
    c->poisoned = false;
    return QS_OK;
}

qs_status qs_step(qs_ctx *c, int n_steps) {
    QS_RANGE("qs_step");
    qs_status s = check_ready(c);
    if (s) return s;
    if (n_steps < 1) return fail(c, QS_ERR_ARG, "n_steps must be >= 1");
    long long max_snap = 0;
    if (c->rec_buf) {
        // number of snapshots this call would write must fit the buffer
        const long long snapd = snapshot_doubles(c, c->rec_kinds);
        max_snap = (long long)(c->rec_bytes / (size_t)(snapd * 8));
        const long long last = c->step + n_steps - 1;
        if (last >= c->rec_g0) {
            const long long d = last - c->rec_g0;
            if (d / c->rec_stride >= max_snap)
                return fail(c, QS_ERR_ARG, "record buffer holds %lld snapshots; this call reaches snapshot %lld",
                            max_snap, d / c->rec_stride);
        }
    }
    s = launch_sweep(c, c->step, n_steps, 1, c->rec_buf ? c->rec_kinds : 0,
                     static_cast<double *>(c->rec_buf), c->rec_g0, c->rec_stride, max_snap);
    if (s) return s;
    c->step += n_steps;
    c->theta_zero = false;
    return QS_OK;
}

qs_status qs_record(qs_ctx *c, int kinds, int stride, void *dev_out, size_t out_bytes) {
    QS_RANGE("qs_record");
    if (!c) return QS_ERR_ARG;
    if (kinds == 0 || !dev_out) {
        c->rec_buf = nullptr; c->rec_kinds = 0; c->rec_bytes = 0;
        return QS_OK;
    }
    if ((kinds & ~7) || stride < 1) return fail(c, QS_ERR_ARG, "record kinds/stride");
    const long long snapd = snapshot_doubles(c, kinds);
    if (out_bytes < (size_t)snapd * 8) return fail(c, QS_ERR_ARG, "record buffer smaller than one snapshot (%lld bytes)", snapd * 8);
    c->rec_kinds = kinds; c->rec_stride = stride; c->rec_buf = dev_out; c->rec_bytes = out_bytes;
    c->rec_g0 = c->step;
    return QS_OK;
}

qs_status qs_diag(qs_ctx *c, int kind, void *out, size_t out_bytes, int out_on_host) {
    QS_RANGE("qs_diag");
    if (!c || !out) return c ? fail(c, QS_ERR_ARG, "null out") : QS_ERR_ARG;
    if (kind == QS_DIAG_STATE) {
        if (!c->seeded) return fail(c, QS_ERR_STATE, "not seeded");
        const size_t need = 64 + c->state_bytes + c->th_bytes + c->ex_bytes;
        if (out_bytes < need) return fail(c, QS_ERR_ARG, "checkpoint needs %zu bytes", need);
        int64_t hdr[8] = {0x51534350, c->prec, c->NS, c->Mp, c->cells_total, c->step, c->groups_total, 1};
        cudaMemcpyKind k = out_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        char *o = static_cast<char *>(out);
        if (out_on_host) memcpy(o, hdr, 64);
        else CU(c, cudaMemcpyAsync(o, hdr, 64, cudaMemcpyHostToDevice, c->stream));
        CU(c, cudaMemcpyAsync(o + 64, c->st, c->state_bytes, k, c->stream));
        if (c->th_bytes) CU(c, cudaMemcpyAsync(o + 64 + c->state_bytes, c->th, c->th_bytes, k, c->stream));
        if (c->ex_bytes) CU(c, cudaMemcpyAsync(o + 64 + c->state_bytes + c->th_bytes, c->ex, c->ex_bytes, k, c->stream));
        CU(c, cudaStreamSynchronize(c->stream));   // hdr lives on this stack frame
        return QS_OK;
    }
    if (kind == QS_DIAG_XIMAX) {
        // field pass into a temporary MAG snapshot, then max over modes per cell
        qs_status s0 = check_ready(c);
        if (s0) return s0;
        const size_t need_x = (size_t)c->cells_total * 3 * sizeof(double);
        if (out_bytes < need_x) return fail(c, QS_ERR_ARG, "diag needs %zu bytes", need_x);
        void *mag = nullptr, *res = nullptr;
        if ((s0 = dalloc(c, (size_t)snapshot_doubles(c, QS_REC_MAG) * 8, &mag))) return s0;
        if (out_on_host && (s0 = dalloc(c, need_x, &res))) return s0;
        double *dres = out_on_host ? static_cast<double *>(res) : static_cast<double *>(out);
        s0 = launch_sweep(c, c->step, 1, 0, QS_REC_MAG, static_cast<double *>(mag), c->step, 1, 1);
        if (!s0) {
            qsk::k_ximax<<<(unsigned)c->cells_total, 256, 0, c->stream>>>(static_cast<const double *>(mag), c->cells_total,
                                                                          c->Mp, c->M, dres);
            cudaError_t e = cudaGetLastError();
            if (!e && out_on_host) e = cudaMemcpyAsync(out, dres, need_x, cudaMemcpyDeviceToHost, c->stream);
            if (!e) e = cudaStreamSynchronize(c->stream);
            if (e) s0 = fail(c, QS_ERR_CUDA, "ximax: %s", cudaGetErrorString(e));
        }
        for (void *p : {mag, res}) {
            if (!p) continue;
            for (size_t i = 0; i < c->bufs.size(); ++i)
                if (c->bufs[i].p == p) {
                    if (c->has_alloc) c->alloc.free(p, c->alloc.user); else cudaFree(p);
                    c->bufs.erase(c->bufs.begin() + i);
                    break;
                }
        }
        return s0 ? s0 : (out_on_host ? qs_sync(c) : QS_OK);
    }
    size_t need;
    double *dst = nullptr;
    if (kind == QS_DIAG_WAKE0) {
        need = (size_t)c->cells_total * 2 * sizeof(double);
    } else if (kind >= 1 && kind <= 7) {
        qs_status s = check_ready(c);
        if (s) return s;
        need = (size_t)snapshot_doubles(c, kind) * 8;
    } else {
        return fail(c, QS_ERR_ARG, "diag kind %d", kind);
    }
    if (out_bytes < need) return fail(c, QS_ERR_ARG, "diag needs %zu bytes", need);
    if (out_on_host) {
        if (c->diag_tmp_bytes < need) {   // grow the staging buffer (rare)
            if (c->diag_tmp) {
                CU(c, cudaStreamSynchronize(c->stream));
                for (size_t i = 0; i < c->bufs.size(); ++i)
                    if (c->bufs[i].p == c->diag_tmp) {
                        if (c->has_alloc) c->alloc.free(c->diag_tmp, c->alloc.user); else cudaFree(c->diag_tmp);
                        c->bufs.erase(c->bufs.begin() + i);
                        break;
                    }
                c->diag_tmp = nullptr;
                c->diag_tmp_bytes = 0;
            }
            qs_status s = dalloc(c, need, &c->diag_tmp);
            if (s) return s;
            c->diag_tmp_bytes = need;
        }
        dst = static_cast<double *>(c->diag_tmp);
    } else {
        dst = static_cast<double *>(out);
    }
    qs_status s = QS_OK;
    if (kind == QS_DIAG_WAKE0) {
        qsk::WakeArgs w{c->inst_d, c->shape_d, c->dens_d, c->n_inst, c->NS, dst};
        qsk::k_wake0<<<(c->n_inst + 63) / 64, 64, 0, c->stream>>>(w);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = fail(c, QS_ERR_CUDA, "wake launch: %s", cudaGetErrorString(e));
    } else {
        s = launch_sweep(c, c->step, 1, 0, kind, dst, c->step, 1, 1);
    }
    if (out_on_host) {
        if (s == QS_OK) {
            cudaError_t e = cudaMemcpyAsync(out, dst, need, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) s = fail(c, QS_ERR_CUDA, "diag copy: %s", cudaGetErrorString(e));
        }
        if (s == QS_OK) s = qs_sync(c);
    }
    return s;
}

qs_status qs_query(const qs_ctx *c, int what, int64_t arg, int64_t *value) {
    if (!c || !value) return QS_ERR_ARG;
    switch (what) {
    case QS_Q_N_MODES: *value = c->M; break;
    case QS_Q_MODES_PADDED: *value = c->Mp; break;
    case QS_Q_N_INST: *value = c->n_inst; break;
    case QS_Q_TOTAL_CELLS: *value = c->cells_total; break;
    case QS_Q_STEP: *value = c->step; break;
    case QS_Q_STATE_BYTES: *value = (int64_t)(64 + c->state_bytes + c->th_bytes + c->ex_bytes); break;
    case QS_Q_SNAPSHOT_BYTES:
        *value = arg == QS_DIAG_XIMAX ? 3 * c->cells_total * 8 : snapshot_doubles(c, (int)arg) * 8;
        break;
    case QS_Q_CELL_OFFSET:
        if (arg < 0 || arg >= c->n_inst) return QS_ERR_ARG;
        *value = c->inst[arg].cell_off;
        break;
    case QS_Q_LAUNCH:
        *value = c->launch.warps_per_cta | (c->launch.prefetch << 8) | (c->launch.persistent << 16) |
                 ((int64_t)c->launch.ctas_per_sm << 24) | ((int64_t)c->launch.variant << 32) |
                 ((int64_t)c->launch.scan_cells << 40);
        break;
    case QS_Q_RES_EVERY: *value = c->res_every; break;
    default: return QS_ERR_ARG;
    }
    return QS_OK;
}

qs_status qs_modes(const qs_ctx *c, double *kx, double *ky) {
    if (!c || !kx || !ky) return QS_ERR_ARG;
    for (int m = 0; m < c->M; ++m) { kx[m] = c->kx[m]; ky[m] = c->ky[m]; }
    return QS_OK;
}

qs_status qs_set_launch(qs_ctx *c, const qs_launch *l) {
    if (!c || !l) return QS_ERR_ARG;
    const int w = l->warps_per_cta;
    if (l->variant < QS_VARIANT_REGISTERS || l->variant > QS_VARIANT_RESIDENT) return fail(c, QS_ERR_ARG, "variant");
    if (l->variant == QS_VARIANT_RESIDENT) {
        if (c->prec != QS_FP32_RENORM) return fail(c, QS_ERR_UNSUPPORTED, "the resident variant is FP32 only");
        if (c->res_every < 1)
            return fail(c, QS_ERR_UNSUPPORTED, "resident: the state may grow by e^%.3g per step, beyond the range "
                        "its FP32 scan partials keep between renormalisations; use a streaming variant", c->growth);
        const int V = l->prefetch;
        if (!res_shape_ok(c->NS, V, w, res_regs(c->NS, V, l->scan_cells)))
            return fail(c, QS_ERR_ARG, "resident: cells per thread 8|16 (any CTA size) or 32 (one species, 2|4|8 "
                                       "warps; Theta in registers: 1|2|4|8); two species: 8 (any) or 16 (4|8|16 "
                                       "warps; Theta in registers: 1|2|4|8)");
        if (res_threads_per_line(max_nxi(c), V) > 32 * w)
            return fail(c, QS_ERR_ARG, "resident: a line of %d cells needs %d threads, the CTA has %d", max_nxi(c),
                        res_threads_per_line(max_nxi(c), V), 32 * w);
        if (l->persistent && (l->ctas_per_sm < 1 || l->ctas_per_sm > 32)) return fail(c, QS_ERR_ARG, "ctas_per_sm");
        c->launch = *l;
        for (auto &g : c->graphs) cudaGraphExecDestroy(g.second);
        c->graphs.clear();
        return QS_OK;
    }
    if (l->variant == QS_VARIANT_SCAN) {
        if (c->prec != QS_FP64) return fail(c, QS_ERR_UNSUPPORTED, "the scan variant is FP64 only");
        const int S = l->prefetch;
        if (!(S == 2 || S == 4 || S == 8 || S == 16 || S == 32) || l->scan_cells < 1 || l->scan_cells > 64 ||
            !(l->warps_per_cta >= 1 && l->warps_per_cta <= 4))
            return fail(c, QS_ERR_ARG, "scan: prefetch = lanes per mode (2..32), scan_cells 1..64, 1..4 warps");
        c->launch = *l;
        for (auto &g : c->graphs) cudaGraphExecDestroy(g.second);
        c->graphs.clear();
        return QS_OK;
    }
    if (!(w == 1 || w == 2 || w == 4 || w == 8)) return fail(c, QS_ERR_ARG, "warps_per_cta");
    const bool f32 = c->prec == QS_FP32_RENORM;
    if (l->variant == QS_VARIANT_TMA) {
        if (f32 ? !(l->prefetch == 8 || l->prefetch == 16) : !(l->prefetch == 4 || l->prefetch == 8))
            return fail(c, QS_ERR_ARG, "TMA tile cells must be 8|16 (FP32) or 4|8 (FP64)");
    } else if (f32 ? !(l->prefetch == 4 || l->prefetch == 8) : !(l->prefetch == 2 || l->prefetch == 4)) {
        return fail(c, QS_ERR_ARG, "prefetch must be 4|8 (FP32) or 2|4 (FP64)");
    }
    if (l->persistent && (l->ctas_per_sm < 1 || l->ctas_per_sm > 64)) return fail(c, QS_ERR_ARG, "ctas_per_sm");
    c->launch = *l;
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.second);
    c->graphs.clear();
    return QS_OK;
}

qs_status qs_get_launch(const qs_ctx *c, qs_launch *l) {
    if (!c || !l) return QS_ERR_ARG;
    *l = c->launch;
    return QS_OK;
}

qs_status qs_sync(qs_ctx *c) {
    QS_RANGE("qs_sync");
    if (!c) return QS_ERR_ARG;
    qs_status cs = check_canaries(c);
    if (cs) return cs;
    int e[4] = {0, 0, 0, 0};
    // on the context's stream: a plain cudaMemcpy would also wait for every
    // other blocking stream of the device
    CU(c, cudaMemcpyAsync(e, c->err_d, sizeof e, cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    if (e[0]) {
        c->poisoned = true;
        if (e[0] & qsk::ERR_CANARY)
            return fail(c, QS_ERR_BOUNDS, "the guard after buffer %d was overwritten (a write past its end)", e[1] - 1);
        if (e[0] & qsk::ERR_BOUNDS) {
            long long bad = 0;
            memcpy(&bad, e + 2, sizeof bad);
            return fail(c, QS_ERR_BOUNDS, "an index left its buffer (bounds-checked build): first bad index %lld",
                        bad - 1);
        }
        if (e[0] & qsk::ERR_TIMEOUT) return fail(c, QS_ERR_TIMEOUT, "a bounded device wait ran out");
        return fail(c, QS_ERR_NONFINITE, "non-finite value in the state");
    }
    return QS_OK;
}

int64_t qs_launch_count(const qs_ctx *c) { return c ? c->n_launch : -1; }

qs_status qs_growth_bound(const qs_params *p, double *efolds_per_step, int *res_every) {
    QS_RANGE("qs_growth_bound");
    if (!p) return QS_ERR_ARG;
    qs_status st = validate(*p, 0);
    if (st) return st;
    std::vector<double> shp;
    if (!profile_shape(*p, shp)) return fail(nullptr, QS_ERR_ARG, "profile");
    double lc = 0.0;
    const double g = qsp::growth_bound(*p, shp, &lc);
    if (efolds_per_step) *efolds_per_step = g;
    if (res_every) *res_every = qsp::res_every_for(g, lc, p->n_xi * p->dxi);
    return QS_OK;
}

qs_status qs_debug_canary(qs_ctx *c, int buffer) {
    if (!c || buffer < 0 || buffer >= (int)c->bufs.size()) return QS_ERR_ARG;
    CU(c, cudaMemsetAsync(static_cast<char *>(c->bufs[buffer].p) + c->bufs[buffer].canary + 7, 0, 1, c->stream));
    return QS_OK;
}

qs_status qs_debug_bounds(qs_ctx *c, int64_t rows_cut) {
    if (!c || rows_cut < 0 || rows_cut > c->cells_total * c->NS) return QS_ERR_ARG;
    c->dbg_rows_cut = rows_cut;
    return QS_OK;
}

int qs_build_flags(void) {
#ifdef QS_CHECK_BOUNDS
    return QS_BUILD_CHECK_BOUNDS;
#else
    return 0;
#endif
}

qs_status qs_debug_waits(qs_ctx *c, int64_t spin_limit, int unsatisfiable) {
    if (!c || spin_limit < 1) return QS_ERR_ARG;
    c->spin_limit = spin_limit;
    c->tx_extra = unsatisfiable ? 16 : 0;
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.second);
    c->graphs.clear();
    return QS_OK;
}

const char *qs_last_error(const qs_ctx *c) { return c ? c->err.c_str() : g_init_err.c_str(); }

}  // extern "C"

// internal (same library): the context's stream and allocator, for the
// surrogate entry points of qs_mlp.cu
cudaStream_t qs_ctx_stream(const qs_ctx *c) { return c ? c->stream : nullptr; }
const qs_allocator *qs_ctx_allocator(const qs_ctx *c) { return c && c->has_alloc ? &c->alloc : nullptr; }

extern "C" {

void qs_free(qs_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.second);
    for (auto &b : c->bufs) {
        if (c->has_alloc) c->alloc.free(b.p, c->alloc.user); else cudaFree(b.p);
    }
    delete c;
}

}  // extern "C"

#include "qs_tune.inc"
#include "qs_green.inc"
#include "qs_surdata.inc"
