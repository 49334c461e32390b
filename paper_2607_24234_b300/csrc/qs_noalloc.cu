// qs_noalloc.cu -- qs_sweep_noalloc: the sweep without any allocation.
//
// Who needs this: callers that may not call cudaMalloc (or any allocating
// routine) at the moment they step the solver -- for example a host
// framework that owns all device memory through its own pool and forbids
// driver allocations in its steady-state loop, or code that must not
// allocate because allocation would synchronise the device or could fail
// mid-run.  Such a caller keeps the state buffers itself and calls this
// entry point; everything else the sweep needs (the per-mode coefficient
// tables, the work list, the persistent-scheduler ticket and the device
// error word) lives in one fixed, file-scope device array.
//
// Properties (also stated in qs.h):
//   - The scratch array is NOALLOC_SCRATCH_BYTES (4 MiB) and is held by
//     every GPU that loads the library, until the process exits.
//   - The first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current); make that first call
//     before any stream capture.
//   - Every call reuses the same array and leaves its contents behind; the
//     ticket and error word are cleared at the start of each call.  Two
//     calls whose work overlaps on the GPU (e.g. on different streams) race
//     on the array.
//   - The tables are built on the host and copied from ordinary (pageable)
//     host memory, so a call may wait for the stream before it returns, and
//     a call on a stream that is being captured is refused
//     (QS_ERR_UNSUPPORTED) before anything is enqueued: a captured copy
//     would read host memory that is gone when the graph runs.
//   - No cudaMalloc, cudaFree or other allocating routine is called.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "qs.h"
#include "qs_nvtx.h"
#include "qs_kernels.cuh"
#include "qs_problem.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices];

// Device address of the scratch array for the current device (looked up
// once per device, with that device current).
qs_status noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return QS_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return QS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) { cudaGetLastError(); return QS_ERR_CUDA; }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return QS_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" qs_status qs_sweep_noalloc(const qs_params *p, void *state, void *theta, int *exponents,
                                      int64_t step0, int n_steps, int *dev_status, void *stream) {
    QS_RANGE("qs_sweep_noalloc");
    // ---- host-side checks (nothing is enqueued on failure) ----
    if (!p || !state || n_steps < 1 || step0 < 0) return QS_ERR_ARG;
    if (p->front == QS_FRONT_HELD) return QS_ERR_UNSUPPORTED;   // held values need a table of their own
    char msg[256];
    qs_status vs = qsp::validate(*p, 0, msg, sizeof msg);
    if (vs) return vs;
    if (p->prec == QS_FP32_RENORM && !exponents) return QS_ERR_ARG;
    if (p->prec == QS_FP64 && !theta) return QS_ERR_ARG;
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs) != cudaSuccess) {
            cudaGetLastError();
            return QS_ERR_CUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) return QS_ERR_UNSUPPORTED;
    }

    // ---- transverse modes and profile (the same definitions as qs_init) ----
    qsp::ModeList modes;
    qsp::build_modes(*p, modes);
    const std::vector<double> &k2 = modes.k2;
    std::vector<double> shape;
    if (!qsp::profile_shape(*p, shape)) return QS_ERR_ARG;
    const int M = (int)k2.size();
    if (M < 1) return QS_ERR_ARG;
    const int Mp = (M + 31) / 32 * 32;
    const int NS = p->n_species;
    const bool f32 = p->prec == QS_FP32_RENORM;
    const int per_item = 64;   // two warps per CTA
    const int n_items = (M + per_item - 1) / per_item;

    // ---- scratch layout and its size limit ----
    const size_t off_ctrl = 0;                                   // ticket, error word
    const size_t off_inst = align256(off_ctrl + 8 * sizeof(int));
    const size_t off_kap = align256(off_inst + sizeof(qsk::InstDev));
    const size_t off_kapk2 = align256(off_kap + sizeof(double) * Mp);
    const size_t off_kabs = align256(off_kapk2 + sizeof(double) * Mp);
    const size_t off_items = align256(off_kabs + sizeof(double) * Mp);
    const size_t off_w = align256(off_items + sizeof(int2) * n_items);
    const size_t w_bytes = (size_t)p->n_xi * NS * (f32 ? sizeof(float) : sizeof(double));
    const size_t total = align256(off_w + w_bytes);
    if (total > NOALLOC_SCRATCH_BYTES) return QS_ERR_ARG;   // beyond the fixed scratch

    void *base = nullptr;
    qs_status st = noalloc_scratch(&base);
    if (st) return st;
    char *sc = static_cast<char *>(base);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // ---- host tables ----
    qsk::InstDev I{};
    I.n_xi = p->n_xi;
    I.n_grp = (p->n_xi + qsk::GRP - 1) / qsk::GRP;
    I.cell_off = 0;
    I.grp_off = 0;
    I.c = std::cos(p->dxi); I.s = std::sin(p->dxi);
    I.ch = std::cos(0.5 * p->dxi); I.sh = std::sin(0.5 * p->dxi);
    I.dt = p->dt; I.dxi = p->dxi;
    const double g = p->gamma_b;
    for (int sp = 0; sp < 2; ++sp) {
        if (sp < NS) {
            const double qm = p->species[sp].q / p->species[sp].m;
            I.q[sp] = p->species[sp].q;
            I.qm_g[sp] = qm / g;
            I.qm_g3[sp] = p->model == QS_MODEL_REDUCED ? 0.0 : qm / (g * g * g);
        }
    }
    std::vector<double> kap(Mp, 1.0), kapk2(Mp, 0.0), kabs(Mp, 0.0);
    for (int m = 0; m < M; ++m) {
        kap[m] = 1.0 / (1.0 + k2[m]);
        kapk2[m] = k2[m] * kap[m];
        kabs[m] = std::sqrt(k2[m]);
    }
    std::vector<int2> items(n_items);
    for (int i = 0; i < n_items; ++i) items[i] = make_int2(0, i * per_item);
    std::vector<double> wd((size_t)p->n_xi * NS);
    for (int j = 0; j < p->n_xi; ++j)
        for (int sp = 0; sp < NS; ++sp) wd[(size_t)j * NS + sp] = p->dt * p->species[sp].density_ratio * shape[j];
    std::vector<float> wf;
    if (f32) wf.assign(wd.begin(), wd.end());

    // ---- enqueue: clear the control words, upload the tables, sweep ----
    // (copies from pageable host memory return once the source is staged)
    auto H2D = [&](size_t off, const void *src, size_t n) {
        return cudaMemcpyAsync(sc + off, src, n, cudaMemcpyHostToDevice, s);
    };
    cudaError_t e = cudaMemsetAsync(sc + off_ctrl, 0, 8 * sizeof(int), s);
    if (!e) e = H2D(off_inst, &I, sizeof I);
    if (!e) e = H2D(off_kap, kap.data(), sizeof(double) * Mp);
    if (!e) e = H2D(off_kapk2, kapk2.data(), sizeof(double) * Mp);
    if (!e) e = H2D(off_kabs, kabs.data(), sizeof(double) * Mp);
    if (!e) e = H2D(off_items, items.data(), sizeof(int2) * n_items);
    if (!e) e = f32 ? H2D(off_w, wf.data(), w_bytes) : H2D(off_w, wd.data(), w_bytes);
    if (e) { cudaGetLastError(); return QS_ERR_CUDA; }

    qsk::SweepArgs a{};
    a.st = state;
    a.th = f32 ? nullptr : theta;
    a.ex = f32 ? exponents : nullptr;
    a.inst = reinterpret_cast<const qsk::InstDev *>(sc + off_inst);
    a.items = reinterpret_cast<const int2 *>(sc + off_items);
    a.n_items = n_items;
    a.kap = reinterpret_cast<const double *>(sc + off_kap);
    a.kapk2 = reinterpret_cast<const double *>(sc + off_kapk2);
    a.kabs = reinterpret_cast<const double *>(sc + off_kabs);
    a.held = nullptr;
    a.w = sc + off_w;
    a.Mp = Mp; a.M = M; a.n_inst = 1;
    a.front = p->front;
    a.step0 = step0; a.n_steps = n_steps; a.update = 1;
    a.persistent = 1;
    a.rec_kinds = 0; a.rec = nullptr;
    a.rows_total = (long long)p->n_xi * NS;
    a.groups_total = I.n_grp;
    a.rec_cap = 0;
    a.res_every = 16;
    a.ticket = reinterpret_cast<int *>(sc + off_ctrl);
    a.err = reinterpret_cast<int *>(sc + off_ctrl) + 4;
    int nsm = 148, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    const dim3 grid((unsigned)std::max(1, std::min(8 * nsm, n_items)));
    if (f32) {
        if (NS == 1) qsk::k_sweep<float, 1, 8, false><<<grid, per_item, 0, s>>>(a);
        else qsk::k_sweep<float, 2, 8, false><<<grid, per_item, 0, s>>>(a);
    } else {
        if (NS == 1) qsk::k_sweep<double, 1, 4, false><<<grid, per_item, 0, s>>>(a);
        else qsk::k_sweep<double, 2, 4, false><<<grid, per_item, 0, s>>>(a);
    }
    if (cudaGetLastError() != cudaSuccess) return QS_ERR_CUDA;
    if (dev_status &&
        cudaMemcpyAsync(dev_status, a.err, sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return QS_ERR_CUDA;
    }
    return QS_OK;
}
