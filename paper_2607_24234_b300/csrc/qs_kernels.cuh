// qs_kernels.cuh -- sm_103a device code of the linearised QSA sweep.
//
// Data layout in HBM (per context, instances concatenated along xi):
//   FP32 path: st  float4 [cell][species][Mp] = (Re n_b, Im n_b, Re Theta, Im Theta)
//              ex  int32  [group][Mp], group = 32 cells: (W << 8) | (s & 0xff)
//                  value = mantissa * 2^W; s = floor(log2(max |mantissa|)) of the
//                  group as written, applied lazily on the next read.
//   FP64 path: st  double2 [cell][species][Mp] = n_b,  th double2 [...] = Theta
// Mp = active modes padded to a multiple of 32, so that a warp touches one
// contiguous 512 B (FP32) / 2 x 512 B (FP64) row per cell and species.
//
// One thread owns one (instance, mode) line and marches it causally in xi
// (Sec. II, Eq. 5, exact per cell with rho constant on the cell), fusing the
// field evaluation (Eq. 14) and the leapfrog push of Eqs. (8)-(9).  Lines are
// independent for all time, so a launch runs all requested slow-time steps
// of its line before taking the next one.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qsk {

constexpr int GRP = 32;          // renormalisation group length (cells)
constexpr int ERR_NONFINITE = 1; // bits of the sticky device error word
constexpr int ERR_TIMEOUT = 2;
constexpr int ERR_BOUNDS = 4;    // bounds-checked build: an index left its buffer (access skipped)
constexpr int ERR_CANARY = 8;    // the guard after a buffer was overwritten

struct InstDev {
    int n_xi, n_grp;
    long long cell_off;   // first cell of this instance in the concatenation
    long long grp_off;    // first exponent group
    double c, s, ch, sh;  // cos, sin of dxi and of dxi/2
    double dt, dxi;
    double q[2];
    double qm_g[2];       // (q/m)/gamma
    double qm_g3[2];      // (q/m)/gamma^3, 0 for the reduced model
    int noise_inst;       // instance word of the noise seed's Philox counter
    float wu[2];          // dt n_bs0 of every cell when the profile is uniform (the FP32 weight)
};

struct SweepArgs {
    void *st;             // state (see above)
    void *th;             // FP64 Theta (null for FP32)
    int *ex;              // FP32 exponents
    const InstDev *inst;
    const int2 *items;    // (instance, first mode) per work item
    int n_items;
    const double *kap;    // 1/(1+k^2)            [Mp]
    const double *kapk2;  // k^2/(1+k^2)          [Mp]
    const double *kabs;   // |k|                  [Mp]
    const double *held;   // [inst][Mp][4] or null
    const void *w;        // dt * n_bs0(xi_j) per cell and species, T [cell][NS]
    int Mp, M, n_inst;
    int front;
    long long step0;
    int n_steps;
    int update;           // 0: field pass only (no state write)
    int persistent;
    // fused record
    int rec_kinds;
    long long rec_g0, rec_max_snap;
    int rec_stride;
    double *rec;
    long long rec_snap_doubles, rec_off_mag, rec_off_np, rec_off_mm, cells_total;
    int *ticket;
    int *err;
    int scan_v;           // scan variant: cells per lane per sub-chunk
    long long spin_limit; // TMA variant: bound on every mbarrier wait (iterations)
    int tx_extra;         // test hook: extra bytes each tile barrier expects (0)
    int res_every;        // resident variant: steps between renormalisation checks (power of two <= 16)
    // extents the bounds-checked build tests every global index against
    long long rows_total;   // state rows: cells_total * NS
    long long groups_total; // exponent-group rows
    long long rec_cap;      // doubles in the record target
};

// Bounds-checked build (QS_CHECK_BOUNDS): chk(a, i, n) is true when 0 <= i <
// n; otherwise it sets ERR_BOUNDS in the error word, keeps the first bad
// index + 1 in words 2..3 of it, and the caller skips the access.  The
// ordinary build compiles every check to `true`.
#ifdef QS_CHECK_BOUNDS
static __device__ __noinline__ bool chk_fail(int *err, long long i) {
    atomicOr(err, ERR_BOUNDS);
    atomicCAS(reinterpret_cast<unsigned long long *>(err + 2), 0ull, (unsigned long long)(i + 1));
    return false;
}
__device__ __forceinline__ bool chk(int *err, long long i, long long n) {
    return (i >= 0 && i < n) ? true : chk_fail(err, i);
}
#define QS_CHK(a, i, n) qsk::chk((a).err, (long long)(i), (long long)(n))
#else
#define QS_CHK(a, i, n) true
#endif

template <typename T> struct Cell { T nr, ni, tr, ti; };

__device__ __forceinline__ float pow2f(int e) {
    if (e < -126) return 0.0f;
    if (e > 127) e = 127;
    return __int_as_float((e + 127) << 23);
}
__device__ __forceinline__ int expof(float x) {   // floor(log2 |x|); -200 for 0 / subnormal
    int b = (__float_as_int(x) >> 23) & 0xff;
    return b ? b - 127 : -200;
}

__device__ __forceinline__ bool cell_ok(const SweepArgs &a, long long row, int mode) {
    return QS_CHK(a, row * a.Mp + mode, a.rows_total * a.Mp) && QS_CHK(a, mode, a.Mp);
}
__device__ __forceinline__ void ld_cell(const SweepArgs &a, long long row, int mode, Cell<float> &c) {
    if (!cell_ok(a, row, mode)) { c.nr = c.ni = c.tr = c.ti = 0.f; return; }
    float4 v = __ldcg(reinterpret_cast<const float4 *>(a.st) + row * a.Mp + mode);
    c.nr = v.x; c.ni = v.y; c.tr = v.z; c.ti = v.w;
}
__device__ __forceinline__ void ld_cell(const SweepArgs &a, long long row, int mode, Cell<double> &c) {
    if (!cell_ok(a, row, mode)) { c.nr = c.ni = c.tr = c.ti = 0.0; return; }
    double2 x = __ldcg(reinterpret_cast<const double2 *>(a.st) + row * a.Mp + mode);
    double2 y = __ldcg(reinterpret_cast<const double2 *>(a.th) + row * a.Mp + mode);
    c.nr = x.x; c.ni = x.y; c.tr = y.x; c.ti = y.y;
}
__device__ __forceinline__ void st_cell(const SweepArgs &a, long long row, int mode, const Cell<float> &c) {
    if (!cell_ok(a, row, mode)) return;
    __stcg(reinterpret_cast<float4 *>(a.st) + row * a.Mp + mode, make_float4(c.nr, c.ni, c.tr, c.ti));
}
__device__ __forceinline__ void st_cell(const SweepArgs &a, long long row, int mode, const Cell<double> &c) {
    if (!cell_ok(a, row, mode)) return;
    __stcg(reinterpret_cast<double2 *>(a.st) + row * a.Mp + mode, make_double2(c.nr, c.ni));
    __stcg(reinterpret_cast<double2 *>(a.th) + row * a.Mp + mode, make_double2(c.tr, c.ti));
}
// exponent word of group row g (FP32 state)
__device__ __forceinline__ int ld_ex(const SweepArgs &a, long long g, int mode) {
    return QS_CHK(a, g * a.Mp + mode, a.groups_total * a.Mp) ? __ldcg(a.ex + g * a.Mp + mode) : 0;
}
__device__ __forceinline__ void st_ex(const SweepArgs &a, long long g, int mode, int v) {
    if (QS_CHK(a, g * a.Mp + mode, a.groups_total * a.Mp)) __stcg(a.ex + g * a.Mp + mode, v);
}

template <typename T> __device__ __forceinline__ double lnabs2(T re2) {  // ln sqrt(re2)
    return 0.5 * log((double)re2);
}

// ---------------------------------------------------------------------------
// Per-line sweep.  U = cells per register batch (divides 32); batches are
// double-buffered so that the loads of batch b+1 are in flight while batch b
// is computed.
// ---------------------------------------------------------------------------
template <typename T, int NS, int U, bool REC>
struct Line {
    static constexpr bool RN = sizeof(T) == 4;   // FP32 path renormalises
    const SweepArgs &a;
    const InstDev &I;
    int inst, mode;
    // plasma state P = (n_p, n_p') entering the current cell, working scale
    T nr, ni, dr, di;
    T c, s, ch, sh, A[NS], B[NS], q[NS];
    T kap, kabsk;          // kappa and |k| kappa (for the fields)
    bool rec, upd;
    long long snap;
    // FP32 renormalisation
    int W, E;              // working scale of the current group, stored scale
    float facM;            // 2^(E - W): stored mantissa -> working scale
    float gmax, gnan;
    double mm0, mm1, mm2;  // running max for MODEMAX (ln of magnitudes)
    double gm0, gm1, gm2;  // running max of squared magnitudes in the current scale

    __device__ Line(const SweepArgs &a_, const InstDev &I_, int inst_, int mode_)
        : a(a_), I(I_), inst(inst_), mode(mode_) {}

    struct Batch { Cell<T> x[U][NS]; T w[U][NS]; int exw; };

    __device__ __forceinline__ void load(Batch &b, int j0) {
        const int N = I.n_xi;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int j = j0 + u;
            if (j < N) {
                long long row = (I.cell_off + j) * NS;
#pragma unroll
                for (int sp = 0; sp < NS; ++sp) {
                    ld_cell(a, row + sp, mode, b.x[u][sp]);
                    b.w[u][sp] = QS_CHK(a, row + sp, a.rows_total) ? __ldg(reinterpret_cast<const T *>(a.w) + row + sp) : T(0);
                }
            }
        }
        if (RN && (j0 % GRP) == 0) b.exw = ld_ex(a, I.grp_off + j0 / GRP, mode);
    }

    __device__ __forceinline__ void group_begin(int exw) {
        if constexpr (RN) {
            E = exw >> 8;
            int s8 = (int)(signed char)(exw & 0xff);
            int Win = E + s8;
            float pm = fmaxf(fmaxf(fabsf((float)nr), fabsf((float)ni)), fmaxf(fabsf((float)dr), fabsf((float)di)));
            int Wn = Win;
            if (pm > 0.0f) { int wp = W + expof(pm); if (wp > Wn) Wn = wp; }
            float facP = pow2f(W - Wn);
            nr *= facP; ni *= facP; dr *= facP; di *= facP;
            W = Wn;
            facM = pow2f(E - W);
            gmax = 0.0f; gnan = 0.0f;
        }
    }

    __device__ __forceinline__ void group_end(int g) {
        if constexpr (RN) {
            if (upd) {
                int s8 = gmax > 0.0f ? expof(gmax) : 0;
                s8 = s8 < -100 ? -100 : (s8 > 100 ? 100 : s8);
                if (!(gnan == 0.0f) || !(gmax <= 3.0e38f)) atomicOr(a.err, ERR_NONFINITE);
                st_ex(a, I.grp_off + g, mode, (W << 8) | (s8 & 0xff));
            }
        }
    }

    __device__ __forceinline__ void record(long long j, T mr, T mi, T mdr, T mdi, T rr, T ri,
                                           const Cell<T> *x) {
        // fields at the cell centre, in the working scale (FP32: x 2^W)
        double nb2 = 0.0;
#pragma unroll
        for (int sp = 0; sp < NS; ++sp)
            nb2 += (double)x[sp].nr * x[sp].nr + (double)x[sp].ni * x[sp].ni;
        const double exr = -(double)kap * mdr, exi = -(double)kap * mdi;
        const double epr = (double)kabsk * ((double)mr - rr), epi = (double)kabsk * ((double)mi - ri);
        const double ex2 = exr * exr + exi * exi;
        const double e2 = ex2 + epr * epr + epi * epi;
        const double kk = (double)kabsk * kabsk;
        const double b2 = kk * ((double)rr * rr + (double)ri * ri);
        if (a.rec_kinds & 3) {
            const double sc = RN ? (double)W * 0.69314718055994530942 : 0.0;
            double *base = a.rec + snap * a.rec_snap_doubles;
            const long long cm = (I.cell_off + j) * a.Mp + mode;
            if ((a.rec_kinds & 1) && QS_CHK(a, cm, a.cells_total * a.Mp) &&
                QS_CHK(a, snap * a.rec_snap_doubles + a.rec_off_mag + cm + 4 * a.cells_total * a.Mp, a.rec_cap)) {
                const long long pl = a.cells_total * a.Mp;
                double *o = base + a.rec_off_mag + cm;
                __stcs(o, 0.5 * log(nb2) + sc);
                __stcs(o + pl, 0.5 * log(e2) + sc);
                __stcs(o + 2 * pl, 0.5 * log(b2) + sc);
                __stcs(o + 3 * pl, 0.5 * log(kk * ((double)mr * mr + (double)mi * mi)) + sc);
                __stcs(o + 4 * pl, 0.5 * log(ex2) + sc);
            }
            if ((a.rec_kinds & 2) && QS_CHK(a, snap * a.rec_snap_doubles + a.rec_off_np + 2 * cm + 1, a.rec_cap)) {
                const double f = RN ? ldexp(1.0, W) : 1.0;
                __stcs(reinterpret_cast<double2 *>(base + a.rec_off_np) + cm,
                       make_double2((double)mr * f, (double)mi * f));
            }
        }
        // per-mode maxima: squared magnitudes within a scale group, one log per group
        if (a.rec_kinds & 4) { gm0 = fmax(gm0, nb2); gm1 = fmax(gm1, e2); gm2 = fmax(gm2, b2); }
    }

    // fold the squared-magnitude maxima of the current scale into the log maxima
    __device__ __forceinline__ void fold_max() {
        if (REC && rec && (a.rec_kinds & 4)) {
            const double sc = RN ? (double)W * 0.69314718055994530942 : 0.0;
            if (gm0 > 0.0) mm0 = fmax(mm0, 0.5 * log(gm0) + sc);
            if (gm1 > 0.0) mm1 = fmax(mm1, 0.5 * log(gm1) + sc);
            if (gm2 > 0.0) mm2 = fmax(mm2, 0.5 * log(gm2) + sc);
            gm0 = gm1 = gm2 = 0.0;
        }
    }

    // One cell: x[NS] holds (n_b, Theta) of cell j as stored (mantissas on
    // the FP32 path), w[NS] = dt n_bs0(xi_j).  Advances P across the cell,
    // records the fields if asked, pushes and stores the beam state.
    __device__ __forceinline__ void cell(Cell<T> *x, const T *w, const int j, const int N) {
        if constexpr (RN) {
#pragma unroll
            for (int sp = 0; sp < NS; ++sp) {
                x[sp].nr *= facM; x[sp].ni *= facM; x[sp].tr *= facM; x[sp].ti *= facM;
            }
        }
        T rr = q[0] * x[0].nr, ri = q[0] * x[0].ni;
        if (NS == 2) { rr = fma(q[NS - 1], x[NS - 1].nr, rr); ri = fma(q[NS - 1], x[NS - 1].ni, ri); }
        if (j == 0 && a.front == 1) { nr = rr; ni = ri; dr = 0; di = 0; }
        // u = n_p - rho; centre:  n_mid = ch u + sh n' + rho
        const T ur = nr - rr, ui = ni - ri;
        const T mr = fma(ch, ur, fma(sh, dr, rr));
        const T mi = fma(ch, ui, fma(sh, di, ri));
        if (REC && rec) {
            const T mdr = fma(-sh, ur, ch * dr), mdi = fma(-sh, ui, ch * di);
            record(j, mr, mi, mdr, mdi, rr, ri, x);
        }
        // cell exit: n = c u + s n' + rho, n' = -s u + c n'
        const T xr = fma(c, ur, fma(s, dr, rr));
        const T xi = fma(c, ui, fma(s, di, ri));
        dr = fma(-s, ur, c * dr);
        di = fma(-s, ui, c * di);
        nr = xr; ni = xi;
        if (upd) {
            const long long row = (I.cell_off + j) * NS;
#pragma unroll
            for (int sp = 0; sp < NS; ++sp) {
                // Theta += h (f1 n_mid - f2 (rho - n_mid));  n_b += dt n_b0 Theta
                x[sp].tr = fma(A[sp], mr, fma(-B[sp], rr, x[sp].tr));
                x[sp].ti = fma(A[sp], mi, fma(-B[sp], ri, x[sp].ti));
                x[sp].nr = fma(w[sp], x[sp].tr, x[sp].nr);
                x[sp].ni = fma(w[sp], x[sp].ti, x[sp].ni);
                if constexpr (RN) {
                    gmax = fmaxf(gmax, fmaxf(fmaxf(fabsf(x[sp].nr), fabsf(x[sp].ni)),
                                             fmaxf(fabsf(x[sp].tr), fabsf(x[sp].ti))));
                    gnan = fmaf(x[sp].nr + x[sp].ti, 0.0f, gnan);
                    gnan = fmaf(x[sp].ni + x[sp].tr, 0.0f, gnan);
                }
                st_cell(a, row + sp, mode, x[sp]);
            }
        }
        if (RN && (((j + 1) % GRP) == 0 || j == N - 1)) {
            fold_max();
            group_end(j / GRP);
        }
    }

    __device__ __forceinline__ void compute(Batch &b, int j0) {
        const int N = I.n_xi;
        if (RN && (j0 % GRP) == 0) group_begin(b.exw);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u;
            if (j < N) cell(b.x[u], b.w[u], j, N);
        }
    }

    // Per-step set-up shared by every kernel variant: slow-time coefficients,
    // record flag and the front boundary value P(0).
    __device__ __forceinline__ void step_begin(int it) {
        const long long g = a.step0 + it;
        const double h = (g == 0) ? 0.5 * I.dt : I.dt;
        const int mk = QS_CHK(a, mode, a.Mp) ? mode : 0;
        const double kapd = a.kap[mk], kk2d = a.kapk2[mk];
#pragma unroll
        for (int sp = 0; sp < NS; ++sp) {
            const double f1 = I.qm_g[sp] * kk2d, f2 = I.qm_g3[sp] * kapd;
            A[sp] = (T)(h * (f1 + f2));
            B[sp] = (T)(h * f2);
            q[sp] = (T)I.q[sp];
        }
        rec = false;
        if (REC) {
            long long d = g - a.rec_g0;
            if (d >= 0 && (d % a.rec_stride) == 0 && d / a.rec_stride < a.rec_max_snap) {
                rec = true;
                snap = d / a.rec_stride;
            }
            mm0 = mm1 = mm2 = -INFINITY;
            gm0 = gm1 = gm2 = 0.0;
        }
        nr = ni = dr = di = 0;
        W = 0;
        if (a.front == 2 && a.held && QS_CHK(a, ((long long)inst * a.Mp + mode) * 4 + 3, (long long)a.n_inst * a.Mp * 4)) {
            const double *hp = a.held + ((long long)inst * a.Mp + mode) * 4;
            if constexpr (RN) {
                double hm = fmax(fmax(fabs(hp[0]), fabs(hp[1])), fmax(fabs(hp[2]), fabs(hp[3])));
                int e = hm > 0.0 ? ilogb(hm) : 0;
                W = e;
                nr = (T)ldexp(hp[0], -e); ni = (T)ldexp(hp[1], -e);
                dr = (T)ldexp(hp[2], -e); di = (T)ldexp(hp[3], -e);
            } else {
                nr = (T)hp[0]; ni = (T)hp[1]; dr = (T)hp[2]; di = (T)hp[3];
            }
        }
    }

    __device__ __forceinline__ void step_end() {
        if (!RN) fold_max();
        if (!(fabs((double)nr) + fabs((double)ni) + fabs((double)dr) + fabs((double)di) <= 1.0e300))
            atomicOr(a.err, ERR_NONFINITE);
        if (REC && rec && (a.rec_kinds & 4) &&
            QS_CHK(a, snap * a.rec_snap_doubles + a.rec_off_mm + ((long long)inst + 2LL * a.n_inst) * a.Mp + mode,
                   a.rec_cap)) {
            double *o = a.rec + snap * a.rec_snap_doubles + a.rec_off_mm + (long long)inst * a.Mp + mode;
            long long pl = (long long)a.n_inst * a.Mp;
            o[0] = mm0; o[pl] = mm1; o[2 * pl] = mm2;
        }
    }

    __device__ __forceinline__ void line_begin() {
        c = (T)I.c; s = (T)I.s; ch = (T)I.ch; sh = (T)I.sh;
        const int mk = QS_CHK(a, mode, a.Mp) ? mode : 0;
        const double kapd = a.kap[mk];
        kap = (T)kapd;
        kabsk = (T)(a.kabs[mk] * kapd);
        upd = a.update != 0;
    }

    __device__ void run() {
        const int N = I.n_xi;
        line_begin();
        for (int it = 0; it < a.n_steps; ++it) {
            step_begin(it);
            Batch b0, b1;
            load(b0, 0);
            for (int j0 = 0; j0 < N; j0 += 2 * U) {
                if (j0 + U < N) load(b1, j0 + U);
                compute(b0, j0);
                if (j0 + 2 * U < N) load(b0, j0 + 2 * U);
                if (j0 + U < N) compute(b1, j0 + U);
            }
            step_end();
        }
    }
};

template <typename T, int NS, int U, bool REC>
__global__ void __launch_bounds__(256) k_sweep(const SweepArgs a) {
    __shared__ int s_item;
    int item = blockIdx.x;
    for (;;) {
        if (a.persistent) {
            if (threadIdx.x == 0) s_item = atomicAdd(a.ticket, 1);
            __syncthreads();
            item = s_item;
            __syncthreads();
        }
        if (item >= a.n_items) break;
        const int2 it = a.items[item];
        const int mode = it.y + threadIdx.x;
        if (mode < a.M) {
            const InstDev I = a.inst[QS_CHK(a, it.x, a.n_inst) ? it.x : 0];
            Line<T, NS, U, REC> L(a, I, it.x, mode);
            L.run();
        }
        if (!a.persistent) break;
    }
}

// ---------------------------------------------------------------------------
// TMA-staged variant.  One warp owns 32 consecutive modes; lane 0 streams
// (xi cells x 32 modes) tiles of the state into shared memory with 2-D
// tensor copies (cp.async.bulk.tensor) through an ST-deep ring of buffers,
// each completing on its own mbarrier; every lane then runs the same
// per-cell arithmetic as k_sweep on its mode and stores the result with
// plain vector stores.  Loads need no registers while in flight, so far more
// bytes are outstanding per SM than with register prefetch.  Every wait is
// bounded: on exhaustion the kernel sets ERR_TIMEOUT, drains its own copies
// (again bounded) and returns.
// ---------------------------------------------------------------------------
namespace tma {
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_bar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void load_2d(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// make this thread's earlier generic-proxy global writes visible to later
// async-proxy (TMA) reads
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
constexpr long long kSpinLimit = 1LL << 24;
}  // namespace tma

template <typename T, int NS, int C, int ST>
__global__ void __launch_bounds__(32) k_sweep_tma(const SweepArgs a, const __grid_constant__ CUtensorMap tmA,
                                                  const __grid_constant__ CUtensorMap tmB) {
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int ROWS = C * NS;
    constexpr int TILE_A = ROWS * 32 * 16;              // float4 / double2 per (row, mode)
    constexpr int TILE = F32 ? TILE_A : 2 * TILE_A;     // FP64: n_b tile then Theta tile
    static_assert(GRP % C == 0, "a chunk never straddles a renormalisation group");
    __shared__ __align__(128) unsigned char buf[ST][TILE];
    __shared__ __align__(8) uint64_t bar[ST];
    const int lane = threadIdx.x;
    if (lane == 0) {
        for (int i = 0; i < ST; ++i) tma::bar_init(&bar[i], 1);
        tma::fence_bar_init();
    }
    __syncwarp();
    uint32_t phase = 0;        // bit i: parity of stage i's next completion
    uint32_t pending = 0;      // bit i: stage i has a copy in flight
    bool dead = false;
    int item = blockIdx.x;
    for (;;) {
        if (a.persistent) {
            int t = 0;
            if (lane == 0) t = atomicAdd(a.ticket, 1);
            item = __shfl_sync(0xffffffffu, t, 0);
        }
        if (item >= a.n_items) break;
        const int2 itx = a.items[item];
        const int mode = itx.y + lane;
        const bool live = mode < a.M;
        const InstDev I = a.inst[QS_CHK(a, itx.x, a.n_inst) ? itx.x : 0];
        Line<T, NS, 1, false> L(a, I, itx.x, live ? mode : itx.y);
        L.line_begin();
        const int N = I.n_xi, nch = (N + C - 1) / C;
        const int x0 = F32 ? itx.y * 4 : itx.y * 2;
        const T *wt = reinterpret_cast<const T *>(a.w) + I.cell_off * NS;
        auto issue = [&](int k) {
            const int stg = k % ST;
            tma::arrive_expect_tx(&bar[stg], TILE + a.tx_extra);
            const int y = (int)((I.cell_off + (long long)k * C) * NS);
            tma::load_2d(buf[stg], &tmA, x0, y, &bar[stg]);
            if (!F32) tma::load_2d(buf[stg] + TILE_A, &tmB, x0, y, &bar[stg]);
        };
        for (int it = 0; it < a.n_steps && !dead; ++it) {
            L.step_begin(it);
            tma::fence_proxy_async();
            __syncwarp();
            if (lane == 0)
                for (int k = 0; k < ST && k < nch; ++k) issue(k);
            for (int k = 0; k < ST && k < nch; ++k) pending |= 1u << k;
            int exn = 0;
            if (F32 && live) exn = ld_ex(a, I.grp_off, mode);
            for (int k = 0; k < nch; ++k) {
                const int stg = k % ST;
                const uint32_t par = (phase >> stg) & 1u;
                long long spins = 0;
                bool ok = tma::try_wait(&bar[stg], par);
                while (!ok && ++spins < a.spin_limit) ok = tma::try_wait(&bar[stg], par);
                if (__any_sync(0xffffffffu, !ok)) { dead = true; break; }
                phase ^= 1u << stg;
                pending &= ~(1u << stg);
                const int j0 = k * C;
                if (live) {
                    if (F32 && (j0 % GRP) == 0) {
                        L.group_begin(exn);
                        if (j0 + GRP < N) exn = ld_ex(a, I.grp_off + (j0 + GRP) / GRP, mode);
                    }
#pragma unroll
                    for (int cc = 0; cc < C; ++cc) {
                        const int j = j0 + cc;
                        if (j < N) {
                            Cell<T> x[NS];
                            T w[NS];
#pragma unroll
                            for (int sp = 0; sp < NS; ++sp) {
                                const int row = cc * NS + sp;
                                if constexpr (F32) {
                                    const float4 v = reinterpret_cast<const float4 *>(buf[stg])[row * 32 + lane];
                                    x[sp].nr = v.x; x[sp].ni = v.y; x[sp].tr = v.z; x[sp].ti = v.w;
                                } else {
                                    const double2 u = reinterpret_cast<const double2 *>(buf[stg])[row * 32 + lane];
                                    const double2 v = reinterpret_cast<const double2 *>(buf[stg] + TILE_A)[row * 32 + lane];
                                    x[sp].nr = u.x; x[sp].ni = u.y; x[sp].tr = v.x; x[sp].ti = v.y;
                                }
                                w[sp] = QS_CHK(a, (I.cell_off + j) * NS + sp, a.rows_total) ? __ldg(wt + (long long)j * NS + sp)
                                                                                           : T(0);
                            }
                            L.cell(x, w, j, N);
                        }
                    }
                }
                __syncwarp();
                if (k + ST < nch) {
                    if (lane == 0) issue(k + ST);
                    pending |= 1u << stg;
                }
            }
            if (!dead && live) L.step_end();
        }
        if (dead || !a.persistent) break;
    }
    if (dead) {
        if (lane == 0) atomicOr(a.err, ERR_TIMEOUT);
        // drain this CTA's own copies before its shared memory is released
        for (int i = 0; i < ST; ++i) {
            if (!(pending & (1u << i))) continue;
            const uint32_t par = (phase >> i) & 1u;
            long long spins = 0;
            while (!tma::try_wait(&bar[i], par) && ++spins < a.spin_limit) {
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Chunked parallel-scan variant (FP64), for problems with few lines.  A warp
// owns MB = 32/S modes; its S lanes per mode split each super-chunk of
// S*V cells into S sub-chunks of V cells.  Pass 1: every lane runs the
// exact cell propagator of Eq. (5) over its V cells from a zero state, which
// gives the affine aggregate B (the transition of V cells is the rotation
// R^V, the same for every lane).  A Hillis-Steele scan over the S lanes of a
// mode (shuffles at distance MB * 2^k, composing with R^(V 2^k)) turns the
// aggregates into each sub-chunk's entry state, R^(V sigma) P_in + sum of
// the earlier aggregates.  Pass 2 re-runs the same per-cell update as
// k_sweep (fields, push, stores) from that entry state; the super-chunk's
// exit state is carried to the next one.
// ---------------------------------------------------------------------------
struct Rot { double c, s; };
__device__ __forceinline__ Rot rot(double ang) { Rot r; sincos(ang, &r.s, &r.c); return r; }
// (n, n') <- R(d) (n, n') for the real and the imaginary parts
__device__ __forceinline__ void rotate(const Rot &R, double &nr, double &ni, double &dr, double &di) {
    const double xr = R.c * nr + R.s * dr, xi = R.c * ni + R.s * di;
    const double yr = -R.s * nr + R.c * dr, yi = -R.s * ni + R.c * di;
    nr = xr; ni = xi; dr = yr; di = yi;
}

template <int NS, int S>
__global__ void __launch_bounds__(128) k_sweep_scan(const SweepArgs a) {
    constexpr int MB = 32 / S;
    const int lane = threadIdx.x & 31;
    const int sig = lane / MB, mm = lane - sig * MB;
    const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= a.n_items) return;                       // uniform per warp
    const int2 itx = a.items[item];
    const int mode = itx.y + mm;
    const bool live = mode < a.M;
    const InstDev I = a.inst[QS_CHK(a, itx.x, a.n_inst) ? itx.x : 0];
    Line<double, NS, 1, false> L(a, I, itx.x, live ? mode : itx.y);
    L.line_begin();
    const int N = I.n_xi, V = a.scan_v, C = S * V;
    const double D = I.dxi;
    const Rot Rsig = rot(D * V * sig), RC = rot(D * C);
    Rot Rlev[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) Rlev[k] = rot(D * V * (1 << k));
    const double c = I.c, s = I.s;
    double q[NS];
#pragma unroll
    for (int sp = 0; sp < NS; ++sp) q[sp] = I.q[sp];
    const double *wt = reinterpret_cast<const double *>(a.w) + I.cell_off * NS;
    for (int it = 0; it < a.n_steps; ++it) {
        L.step_begin(it);
        double Pr = L.nr, Pi = L.ni, Qr = L.dr, Qi = L.di;   // super-chunk entry state
        if (a.front == 1 && live) {
            double rr = 0, ri = 0;
            for (int sp = 0; sp < NS; ++sp) {
                Cell<double> x;
                ld_cell(a, I.cell_off * NS + sp, mode, x);
                rr = fma(q[sp], x.nr, rr);
                ri = fma(q[sp], x.ni, ri);
            }
            Pr = rr; Pi = ri; Qr = 0; Qi = 0;
        }
        for (int J = 0; J < N; J += C) {
            const int j0 = J + sig * V;
            // pass 1: aggregate of this lane's V cells from a zero state
            double br = 0, bi = 0, er = 0, ei = 0;
            for (int v = 0; v < V; ++v) {
                const int j = j0 + v;
                if (j >= N || !live) break;
                double rr = 0, ri = 0;
                for (int sp = 0; sp < NS; ++sp) {
                    const long long cix = ((I.cell_off + j) * NS + sp) * a.Mp + mode;
                    const double2 x = QS_CHK(a, cix, a.rows_total * a.Mp)
                                          ? __ldcg(reinterpret_cast<const double2 *>(a.st) + cix)
                                          : make_double2(0.0, 0.0);
                    rr = fma(q[sp], x.x, rr);
                    ri = fma(q[sp], x.y, ri);
                }
                const double ur = br - rr, ui = bi - ri;
                const double xr = fma(c, ur, fma(s, er, rr)), xi = fma(c, ui, fma(s, ei, ri));
                er = fma(-s, ur, c * er);
                ei = fma(-s, ui, c * ei);
                br = xr; bi = xi;
            }
            // inclusive scan over the S lanes of this mode
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int d = 1 << k;
                if (d >= S) break;
                double ur = __shfl_up_sync(0xffffffffu, br, d * MB), ui = __shfl_up_sync(0xffffffffu, bi, d * MB);
                double vr = __shfl_up_sync(0xffffffffu, er, d * MB), vi = __shfl_up_sync(0xffffffffu, ei, d * MB);
                if (sig >= d) {
                    rotate(Rlev[k], ur, ui, vr, vi);
                    br += ur; bi += ui; er += vr; ei += vi;
                }
            }
            // exclusive prefix, entry state, and the chunk's exit aggregate
            double xr = __shfl_up_sync(0xffffffffu, br, MB), xi = __shfl_up_sync(0xffffffffu, bi, MB);
            double yr = __shfl_up_sync(0xffffffffu, er, MB), yi = __shfl_up_sync(0xffffffffu, ei, MB);
            if (sig == 0) { xr = xi = yr = yi = 0; }
            const int last = (S - 1) * MB + mm;
            const double Br = __shfl_sync(0xffffffffu, br, last), Bi = __shfl_sync(0xffffffffu, bi, last);
            const double Er = __shfl_sync(0xffffffffu, er, last), Ei = __shfl_sync(0xffffffffu, ei, last);
            double nr = Pr, ni = Pi, dr = Qr, di = Qi;
            rotate(Rsig, nr, ni, dr, di);
            L.nr = nr + xr; L.ni = ni + xi; L.dr = dr + yr; L.di = di + yi;
            // pass 2: the real per-cell update
            for (int v = 0; v < V; ++v) {
                const int j = j0 + v;
                if (j >= N || !live) break;
                Cell<double> x[NS];
                double w[NS];
                for (int sp = 0; sp < NS; ++sp) {
                    ld_cell(a, (I.cell_off + j) * NS + sp, mode, x[sp]);
                    w[sp] = QS_CHK(a, (I.cell_off + j) * NS + sp, a.rows_total) ? __ldg(wt + (long long)j * NS + sp) : 0.0;
                }
                L.cell(x, w, j, N);
            }
            rotate(RC, Pr, Pi, Qr, Qi);
            Pr += Br; Pi += Bi; Qr += Er; Qi += Ei;
        }
        if (live) L.step_end();
    }
}

// ---------------------------------------------------------------------------
// Seeds.  Philox4x32-10 (Salmon et al., SC'11) written from its definition.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ void normal2(uint64_t seed, uint32_t j, uint32_t id, uint32_t inst,
                                        uint32_t sp, double &g1, double &g2) {
    uint32_t c[4] = {j, id, inst, sp};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t m1 = ((uint64_t)c[0] << 21) | (c[1] >> 11);
    const uint64_t m2 = ((uint64_t)c[2] << 21) | (c[3] >> 11);
    const double u1 = ((double)m1 + 0.5) * 0x1.0p-53;
    const double u2 = ((double)m2 + 0.5) * 0x1.0p-53;
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    g1 = r * cs;
    g2 = r * sn;
}

struct SeedArgs {
    void *st, *th;
    int *ex;
    const InstDev *inst;
    const double *shape;      // [cell]
    const double *dens;       // [inst][2]
    const int *mode_id, *partner_id;
    int Mp, M, NS, n_inst;
    int kind;                 // 0 noise, 1 impulse, 2 user
    uint64_t seed;
    double amp;
    const double *user;       // complex128 [inst][mode][species][xi]
    long long total_groups;
};

// One thread per (group of 32 cells, mode): writes n_b, Theta and (FP32) the
// group exponent.  Values are formed in FP64.
template <typename T>
__global__ void k_seed(const SeedArgs a) {
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;
    const long long gg = blockIdx.y + (long long)blockIdx.z * gridDim.y;   // global group
    if (mode >= a.Mp || gg >= a.total_groups) return;
    int lo = 0, hi = a.n_inst - 1;             // last instance with grp_off <= gg
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.inst[mid].grp_off <= gg) lo = mid; else hi = mid - 1;
    }
    const int inst = lo;
    const InstDev I = a.inst[inst];
    const int g = (int)(gg - I.grp_off);
    const int j0 = g * GRP, j1 = min(I.n_xi, j0 + GRP);
    const bool live = mode < a.M;
    double v[GRP][2][4];
    double vmax = 0.0;
    for (int j = j0; j < j1; ++j) {
        for (int sp = 0; sp < a.NS; ++sp) {
            double nr = 0, ni = 0, tr = 0, ti = 0;
            if (live) {
                if (a.kind == 0) {
                    const int id = a.mode_id[mode], pid = a.partner_id[mode];
                    const bool cj = pid < id;
                    double g1, g2;
                    normal2(a.seed, (uint32_t)j, (uint32_t)(cj ? pid : id), (uint32_t)I.noise_inst, (uint32_t)sp, g1,
                            g2);
                    const double am = a.amp * a.shape[I.cell_off + j] * 0.70710678118654752440;
                    nr = am * g1;
                    ni = cj ? -am * g2 : am * g2;
                } else if (a.kind == 1) {
                    if (j == 0 && sp == 0)
                        tr = a.amp / (I.q[0] * a.dens[2 * inst] * a.shape[I.cell_off] * I.dxi);
                } else {
                    const long long o = ((((long long)0 + mode) * a.NS + sp) * I.n_xi + j);
                    // user rows are per instance: [inst][mode][sp][xi]
                    const double *ub = a.user + 2 * ((long long)a.M * a.NS * I.cell_off);
                    nr = ub[2 * o];
                    ni = ub[2 * o + 1];
                }
            }
            v[j - j0][sp][0] = nr; v[j - j0][sp][1] = ni; v[j - j0][sp][2] = tr; v[j - j0][sp][3] = ti;
            vmax = fmax(vmax, fmax(fmax(fabs(nr), fabs(ni)), fmax(fabs(tr), fabs(ti))));
        }
    }
    int E = 0;
    if (sizeof(T) == 4 && vmax > 0.0) E = ilogb(vmax);
    for (int j = j0; j < j1; ++j) {
        for (int sp = 0; sp < a.NS; ++sp) {
            const long long row = (I.cell_off + j) * a.NS + sp;
            const double *x = v[j - j0][sp];
            if constexpr (sizeof(T) == 4) {
                reinterpret_cast<float4 *>(a.st)[row * a.Mp + mode] =
                    make_float4((float)ldexp(x[0], -E), (float)ldexp(x[1], -E),
                                (float)ldexp(x[2], -E), (float)ldexp(x[3], -E));
            } else {
                reinterpret_cast<double2 *>(a.st)[row * a.Mp + mode] = make_double2(x[0], x[1]);
                reinterpret_cast<double2 *>(a.th)[row * a.Mp + mode] = make_double2(x[2], x[3]);
            }
        }
    }
    if (sizeof(T) == 4) a.ex[(I.grp_off + g) * a.Mp + mode] = (E << 8);
}

// Per-xi maxima over the active modes of ln|dn_b|, ln|dE|, ln|dB| from a MAG
// snapshot [5][cells][Mp]: one CTA per cell.  out [3][cells].
static __global__ void k_ximax(const double *mag, long long cells, int Mp, int M, double *out) {
    const long long cell = blockIdx.x;
    __shared__ double red[3][256];
    double m0 = -INFINITY, m1 = -INFINITY, m2 = -INFINITY;
    const long long plane = cells * Mp;
    for (int mo = threadIdx.x; mo < M; mo += blockDim.x) {
        const long long o = cell * Mp + mo;
        m0 = fmax(m0, mag[o]);
        m1 = fmax(m1, mag[o + plane]);
        m2 = fmax(m2, mag[o + 2 * plane]);
    }
    red[0][threadIdx.x] = m0; red[1][threadIdx.x] = m1; red[2][threadIdx.x] = m2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = fmax(red[k][threadIdx.x], red[k][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out[k * cells + cell] = red[k][0];
}

// Zeroth-order wake per instance (Eq. 5 with the unperturbed beam charge).
struct WakeArgs {
    const InstDev *inst;
    const double *shape, *dens;
    int n_inst, NS;
    double *out;   // [cell][2] (exit, centre)
};
static __global__ void k_wake0(const WakeArgs a) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= a.n_inst) return;
    const InstDev I = a.inst[inst];
    double n = 0.0, d = 0.0;
    for (int j = 0; j < I.n_xi; ++j) {
        double r = 0.0;
        for (int sp = 0; sp < a.NS; ++sp) r += I.q[sp] * a.dens[2 * inst + sp] * a.shape[I.cell_off + j];
        const double u = n - r;
        const double m = fma(I.ch, u, fma(I.sh, d, r));
        const double x = fma(I.c, u, fma(I.s, d, r));
        d = fma(-I.s, u, I.c * d);
        n = x;
        a.out[2 * (I.cell_off + j)] = n;
        a.out[2 * (I.cell_off + j) + 1] = m;
    }
}

}  // namespace qsk
