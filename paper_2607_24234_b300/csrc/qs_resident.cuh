// qs_resident.cuh -- on-chip ("resident") FP32 sweep, included after
// qs_kernels.cuh.
//
// Lines (instance, transverse mode) never couple (Eq. 14 is diagonal in k),
// so a line can stay on chip for every slow-time step of a launch.  Tl
// threads (whole warps) hold one line: thread t keeps cells [tV, tV + V) of
// every species in registers, and HBM is read when the launch starts and
// written when it ends, nothing in between.  A CTA of T threads holds T / Tl
// lines of one instance (consecutive modes).
//
// Within a step the causal xi march of Eq. (5) becomes a scan.  The exact
// cell propagator is affine in the plasma state P = (n_p, dn_p/dxi):
// P -> R P + rho (1 - cos dxi, sin dxi), R the rotation by dxi.  A chunk of V
// cells therefore maps P to R^V P + A, with A the chunk's response from
// P = 0 (pass 1).  A Hillis-Steele scan over the lanes of a warp (shuffles
// at distance 2^k, composing with R^(V 2^k)) and a sequential pass over the
// line's earlier warps (shared memory, R^(32 V) between warps) give every
// chunk its entry state.  Pass 2 then runs the per-cell update of the
// streaming kernels from that state: fields at the cell centre, the
// leapfrog push of Eqs. (8)-(9).
//
// FP32 range.  Each thread stores its chunk as mantissas times 2^e, one
// exponent per thread; scan partials move between threads' scales by exact
// powers of two.  Every a.res_every-th step a thread renormalises its chunk
// when the largest mantissa has left [2^-16, 2^16], and no exponent of a
// line may lie more than RES_SPAN below the line's largest (checked every
// step).  A scan partial is then at most about 2^(16 + 5) G times
// 2^RES_SPAN in any thread's scale, G the growth between two checks, so
// nothing overflows while G < 2^(128 - 21 - RES_SPAN) = 2^43.  The host
// picks res_every (a power of two up to 16) from a bound of the scheme's
// growth per step derived from the problem statement (qsp::growth_bound),
// so that G stays below e^28; problems whose bound leaves no interval are
// not run by this kernel.  Only values below ~2^-(RES_SPAN + 126) of the
// line maximum flush to zero.
// On the way out the threads sharing a 32-cell group agree on one exponent
// and write the usual (mantissa, exponent word) layout.
#pragma once
#include <type_traits>

namespace qsk {

constexpr int RES_MAX_WARPS = 16;   // T <= 512
constexpr int RES_SPAN = 64;
constexpr int RES_HYST = 16;
constexpr int RES_NONE = -(1 << 20);   // exponent of a thread that holds no value yet
constexpr int RES_REGS64 = 128;       // register cap of the 64-thread shared-Theta kernel (96..224 measured: 128 best)

// register cap per instantiation: 32 cells of state per thread with Theta in
// registers (V NS = 32, TT = 0) need the whole file (no spills at 255; the
// CTA then has at most 256 threads)
constexpr int res_maxnreg(int NS, int V, int TT) { return TT == 64 ? RES_REGS64 : (TT == 0 && V * NS == 32 ? 255 : 128); }

struct RotF { float c, s; };
__device__ __forceinline__ RotF rotf(double ang) {
    double sn, cs;
    sincos(ang, &sn, &cs);
    return RotF{(float)cs, (float)sn};
}
// (n, n') += f R^m (x, x'), real and imaginary parts, R^m = [[C, S], [-S, C]]
__device__ __forceinline__ void acc_rot(float &nr, float &ni, float &dr, float &di, const RotF R, const float f,
                                        const float xr, const float xi, const float yr, const float yi) {
    const float C = R.c * f, S = R.s * f;
    nr = fmaf(C, xr, fmaf(S, yr, nr));
    ni = fmaf(C, xi, fmaf(S, yi, ni));
    dr = fmaf(-S, xr, fmaf(C, yr, dr));
    di = fmaf(-S, xi, fmaf(C, yi, di));
}
// packed (re, im) arithmetic: one f32x2 instruction for both components,
// each rounded as its scalar counterpart (__fmaf_rn, __fmul_rn, __fadd_rn)
__device__ __forceinline__ float2 F2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// (n, n') += f R^m (x, x') with both components of each in one register pair
__device__ __forceinline__ void acc_rot2(float2 &n, float2 &d, const RotF R, const float f, const float2 x,
                                         const float2 y) {
    const float C = R.c * f, S = R.s * f;
    n = pfma(F2(C), x, pfma(F2(S), y, n));
    d = pfma(F2(-S), x, pfma(F2(C), y, d));
}
__device__ __forceinline__ int clamp_shift(int s) { return s < -126 ? -126 : (s > 126 ? 126 : s); }
// 2^e for e in [-126, 127]; 0 below (branch free)
__device__ __forceinline__ float p2(int e) { return __int_as_float((max(-127, min(e, 127)) + 127) << 23); }

// TT > 0 keeps Theta in shared memory (float2 rows [v * NS + sp][thread],
// read and written once per cell in pass 2, next to float rows of the
// weights dt n_b0) so that 32 cells of one species, or 16 of two, fit a
// 128-register budget; the CTA then has exactly TT threads (compile-time row
// stride).  TT = 0 keeps Theta in registers and only the weights in shared
// memory, as (w, w) pairs in rows [v * NS + sp][thread] of the CTA's size,
// so that each cell's weight is one 8-byte load already in the packed form.
// UW (uniform profile in every instance; the host checks): the weight of
// every cell is the instance's I.wu, held in a register pair, with no
// per-cell load.  Cells past the end of a line then carry the weight too and
// evolve, which changes nothing that is kept: xi is causal, so they feed
// only later cells, all of them past the end; they are never written back;
// and threads with no cell of the line keep the sentinel exponent, so the
// line's largest exponent is unaffected.  The one thread that holds the
// line's end counts its padding cells in its renormalisation check, so with
// such lines the results equal the per-cell-weight kernel's to rounding, and
// bit for bit when lines fill whole warps.
template <int NS, int V, int TT, bool UW = false>
__global__ void __maxnreg__(res_maxnreg(NS, V, TT)) k_sweep_res(const SweepArgs a) {
    static_assert(!UW || TT > 0, "a uniform weight replaces the shared-memory weight rows");
    constexpr bool THS = TT > 0;
    static_assert(GRP % V == 0, "a thread's cells lie in one exponent group");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int CB = 2;                     // cells per shared-memory batch (THS; 4 and 8 measured 0.7 % and 0.3 % slower)
    static_assert(V % CB == 0, "whole batches");
    extern __shared__ float4 sdyn[];          // THS: Theta then w, rows [v * NS + sp][T]; else (w, w) [v * NS + sp][T]
    __shared__ float4 sZ[2][RES_MAX_WARPS];   // inclusive warp aggregate (lane 31)
    __shared__ int sE[2][RES_MAX_WARPS];      // its exponent
    __shared__ int sM[2][RES_MAX_WARPS];      // largest exponent in the warp
    __shared__ int s_item;
    __shared__ float2 sRk[6];                 // R^(V 2^k), k = 0..4, and R^(32 V)
    __shared__ float2 sRl[32];                // R^(V lane)
    __shared__ double sMM[RES_MAX_WARPS][3];  // per-warp log maxima of a recording step
    __shared__ float4 sG[32];                 // R^(V-1-v) (1 - cos dxi, sin dxi), each component twice
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = THS ? TT : (int)blockDim.x, nw = T >> 5;
    float2 *sT = reinterpret_cast<float2 *>(sdyn) + tid;                      // THS: row stride T = TT
    float *sWt = reinterpret_cast<float *>(reinterpret_cast<float2 *>(sdyn) + V * NS * (THS ? TT : 0)) + tid;
    float2 *sWr = reinterpret_cast<float2 *>(sdyn) + tid;                     // !THS: row stride T
    int item = blockIdx.x;
    int buf = 0;
    for (;;) {
        if (a.persistent) {
            if (tid == 0) s_item = atomicAdd(a.ticket, 1);
            __syncthreads();
            item = s_item;
            __syncthreads();
        }
        if (item >= a.n_items) break;                  // uniform over the CTA
        const int2 itx = a.items[item];
        const InstDev I = a.inst[QS_CHK(a, itx.x, a.n_inst) ? itx.x : 0];
        const int N = I.n_xi;
        const int Tl = (((N + V - 1) / V) + 31) & ~31;  // threads per line (whole warps)
        const int L = T / Tl;                          // lines per CTA (host: >= 1)
        const int slot = tid / Tl, t = tid - slot * Tl;
        const int mode = itx.y + slot;
        const bool live = slot < L && mode < a.M;
        const int mc = live ? mode : itx.y;
        const int w0 = (slot * Tl) >> 5;
        const int wend = min(w0 + (Tl >> 5), nw);
        const int jb = t * V;
        const bool has = live && jb < N;
        const bool front1 = a.front == 1 && live && t == 0;

        // per-line constants
        const int mk = QS_CHK(a, mc, a.Mp) ? mc : 0;
        const double kapd = a.kap[mk], kk2d = a.kapk2[mk];
        float Af[NS], Bf[NS], q[NS];
#pragma unroll
        for (int sp = 0; sp < NS; ++sp) {
            // the chunk holds y_s = q_s n_bs and q_s Theta_s (exact for |q| a
            // power of two), so rho = sum_s y_s and the kick carries q_s
            const double f1 = I.qm_g[sp] * kk2d, f2 = I.qm_g3[sp] * kapd;
            Af[sp] = (float)(I.q[sp] * (I.dt * (f1 + f2)));
            Bf[sp] = (float)(I.q[sp] * (I.dt * f2));
            q[sp] = (float)I.q[sp];
        }
        const float c = (float)I.c, s = (float)I.s, ch = (float)I.ch, sh = (float)I.sh;
        [[maybe_unused]] float2 W2[NS];
#pragma unroll
        for (int sp = 0; sp < NS; ++sp) W2[sp] = make_float2(I.wu[sp], I.wu[sp]);
        // rotation tables: registers when Theta is in registers, else shared
        // by the CTA's lines (one instance per item; visible after the first
        // barrier below)
        RotF Rk[THS ? 1 : 5], Rl{1.f, 0.f}, Rw{1.f, 0.f};
        if constexpr (!THS) {
#pragma unroll
            for (int k = 0; k < 5; ++k) Rk[k] = rotf(I.dxi * (double)(V << k));
            Rl = rotf(I.dxi * (double)(V * lane));
            Rw = rotf(I.dxi * (double)(32 * V));
        }
        if (THS && warp == 0) {
            const RotF r = rotf(I.dxi * (double)(V * lane));
            sRl[lane] = make_float2(r.c, r.s);
            if (lane < 6) {
                const RotF q6 = rotf(I.dxi * (double)(lane < 5 ? V << lane : 32 * V));
                sRk[lane] = make_float2(q6.c, q6.s);
            }
        }
        if (warp == 0 && lane < V) {
            // a chunk's response from P = 0 is sum_v rho_v R^(V-1-v) g with
            // g = (1 - cos dxi, sin dxi) (Eq. 5 unrolled over the chunk)
            double sn, cs;
            sincos(I.dxi * (double)(V - 1 - lane), &sn, &cs);
            const double sh1 = sin(0.5 * I.dxi), g1 = 2.0 * sh1 * sh1, g2 = I.s;
            const float ga = (float)(cs * g1 + sn * g2), gb = (float)(cs * g2 - sn * g1);
            sG[lane] = make_float4(ga, ga, gb, gb);
        }
        const bool held = a.front == 2 && a.held != nullptr && live && t == 0 &&
                          QS_CHK(a, ((long long)itx.x * a.Mp + mc) * 4 + 3, (long long)a.n_inst * a.Mp * 4);
        const double *hp = held ? a.held + ((long long)itx.x * a.Mp + mc) * 4 : nullptr;

        // load the chunk: mantissas relative to e = W + s8 of its group; cells
        // past the end of the line hold zeros (state and weight)
        float2 xn[V][NS];                      // q_s n_bs (re, im)
        float2 xt[THS ? 1 : V][NS];            // q_s Theta_s when it stays in registers
        int e = RES_NONE;
        float fin = 1.0f;
        if (has) {
            const int exw = ld_ex(a, I.grp_off + jb / GRP, mode);
            const int s8 = (int)(signed char)(exw & 0xff);
            e = (exw >> 8) + s8;
            fin = p2(-s8);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int j = jb + v;
#pragma unroll
            for (int sp = 0; sp < NS; ++sp) {
                float wv = 0.f;
                Cell<float> y{0.f, 0.f, 0.f, 0.f};
                if (has && j < N) {
                    const long long row = (I.cell_off + j) * NS + sp;
                    ld_cell(a, row, mode, y);
                    const float f = fin * q[sp];
                    y.nr *= f; y.ni *= f; y.tr *= f; y.ti *= f;
                    if constexpr (!UW)
                        wv = QS_CHK(a, row, a.rows_total) ? __ldg(reinterpret_cast<const float *>(a.w) + row) : 0.f;
                }
                xn[v][sp] = make_float2(y.nr, y.ni);
                if constexpr (THS) {
                    sT[(v * NS + sp) * T] = make_float2(y.tr, y.ti);
                    if constexpr (!UW) sWt[(v * NS + sp) * T] = wv;
                } else {
                    xt[v][sp] = make_float2(y.tr, y.ti);
                    sWr[(v * NS + sp) * T] = make_float2(wv, wv);   // only this thread reads it back
                }
            }
        }
        auto scale_chunk = [&](float f) {
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
                for (int sp = 0; sp < NS; ++sp) {
                    xn[v][sp].x *= f; xn[v][sp].y *= f;
                    if constexpr (THS) {
                        float2 &z = sT[(v * NS + sp) * T];
                        z.x *= f; z.y *= f;
                    } else {
                        xt[v][sp].x *= f; xt[v][sp].y *= f;
                    }
                }
        };
        if (held) {   // the held front value enters thread 0's scale
            const double hm = fmax(fmax(fabs(hp[0]), fabs(hp[1])), fmax(fabs(hp[2]), fabs(hp[3])));
            if (hm > 0.0) {
                const int eh = ilogb(hm);
                if (eh > e) { scale_chunk(p2(e - eh)); e = eh; }
            }
        }
        // initial clamp to the line maximum
        {
            const int wm = __reduce_max_sync(FULL, e);
            if (lane == 0) sM[buf][warp] = wm;
            __syncthreads();
            int Em = RES_NONE;
            for (int ww = w0; ww < wend; ++ww) Em = max(Em, sM[buf][ww]);
            const int lo = Em - RES_SPAN;
            if (e < lo) { scale_chunk(p2(e - lo)); e = lo; }
            buf ^= 1;
        }
        auto rho = [&](int v) -> float2 { return NS == 2 ? padd(xn[v][0], xn[v][NS - 1]) : xn[v][0]; };
        // front: P entering cell 0 (thread 0 of the line), in this thread's scale
        auto front_state = [&](float2 &n, float2 &d) {
            n = d = F2(0.f);
            if (held) {
                n = make_float2((float)ldexp(hp[0], -e), (float)ldexp(hp[1], -e));
                d = make_float2((float)ldexp(hp[2], -e), (float)ldexp(hp[3], -e));
            }
            if (front1) n = rho(0);   // equilibrium front: n_p = rho, n_p' = 0 at xi = 0
        };
        const float2 C2 = F2(c), S2 = F2(s), M1 = F2(-1.f);

        // exact cell propagator of Eq. (5): u = n - rho, n <- c u + s n' + rho,
        // n' <- -s u + c n'
        auto cross = [&](float2 &n, float2 &d, const float2 u, const float2 r) {
            n = pfma(C2, u, pfma(S2, d, r));
            d = pfma(S2, make_float2(-u.x, -u.y), pmul(C2, d));   // -s u, without a (-s, -s) register pair
        };
        // the front's share R^V P_front of a chunk aggregate (thread 0 of a
        // line with an equilibrium or held front; P_front in this scale)
        auto add_front = [&](float2 &an, float2 &ad) {
            if (front1 || held) {
                float2 pn, pd;
                front_state(pn, pd);
                RotF RV;
                if constexpr (THS) { const float2 r2 = sRk[0]; RV = RotF{r2.x, r2.y}; } else { RV = Rk[0]; }
                acc_rot2(an, ad, RV, 1.0f, pn, pd);
            }
        };
        // pass 1: the chunk's response from its entry state, in closed form:
        // sum_v rho_v G_v, then the front's share; the same operations, in the
        // same order, as the aggregate that pass 2 forms for the next step, so
        // that splitting a run into calls changes no bits (cells past the end
        // hold rho = 0)
        auto pass1 = [&](float2 &an, float2 &ad) {
            an = ad = F2(0.f);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float2 r = rho(v);
                const float4 g = sG[v];
                an = pfma(make_float2(g.x, g.y), r, an);
                ad = pfma(make_float2(g.z, g.w), r, ad);
            }
            add_front(an, ad);
        };
        // pass 2: fields at the cell centre and the push, Theta += A n_mid -
        // B rho, n_b += dt n_b0 Theta; one species folds n_mid = ch u + sh n' +
        // rho into the coefficients (Ach u + Ash n' + (A - B) rho).  GM: track
        // the chunk's largest magnitude for the renormalisation.
        // REC: also the per-mode maxima of |n_b|^2, |E|^2 = kappa^2 |n_p'|^2 +
        // k^2 kappa^2 |n_p - rho|^2 and |B|^2 = k^2 kappa^2 |rho|^2 at the cell
        // centres, before the push (the fields of Eq. 14).  UPD = false: fields
        // only, the state is not changed.
        // UPD also accumulates the NEXT step's chunk aggregate (pass 1 of step
        // k+1) from the pushed rho in its closed form sum_v rho_v G_v (two
        // packed FMAs per cell); the front's share is added after the pass.
        auto pass2 = [&](auto gm_tag, auto rec_tag, auto upd_tag, float2 n, float2 d, const float *A,
                         const float *B, float *mx, const float *rc, float2 &an, float2 &ad) {
            constexpr bool GM = decltype(gm_tag)::value;
            constexpr bool REC = decltype(rec_tag)::value;
            constexpr bool UPD = decltype(upd_tag)::value;
            float gmax = 0.f;
            const float2 Ach = F2(A[0] * ch), Ash = F2(A[0] * sh), AB = F2(A[0] - B[0]);
            const float2 CH2 = F2(ch), SH2 = F2(sh);
            // THS: the Theta and w rows of a batch are loaded one batch ahead
            // (software pipelining), so a batch's shared-memory latency is
            // covered by the previous batch's arithmetic
            [[maybe_unused]] float2 pt[THS ? CB : 1][NS];
            [[maybe_unused]] float pw[THS ? CB : 1][NS];
            if constexpr (THS) {
#pragma unroll
                for (int u = 0; u < CB; ++u)
#pragma unroll
                    for (int sp = 0; sp < NS; ++sp) {
                        pt[u][sp] = sT[(u * NS + sp) * T];
                        if constexpr (!UW) pw[u][sp] = sWt[(u * NS + sp) * T];
                    }
            }
#pragma unroll
            for (int vb = 0; vb < V; vb += CB) {
                float2 zt[THS ? CB : 1][NS];
                [[maybe_unused]] float zw[THS ? CB : 1][NS];
                if constexpr (THS) {
#pragma unroll
                    for (int u = 0; u < CB; ++u)
#pragma unroll
                        for (int sp = 0; sp < NS; ++sp) {
                            zt[u][sp] = pt[u][sp];
                            if constexpr (!UW) zw[u][sp] = pw[u][sp];
                        }
                    if (vb + CB < V) {
#pragma unroll
                        for (int u = 0; u < CB; ++u)
#pragma unroll
                            for (int sp = 0; sp < NS; ++sp) {
                                pt[u][sp] = sT[((vb + CB + u) * NS + sp) * T];
                                if constexpr (!UW) pw[u][sp] = sWt[((vb + CB + u) * NS + sp) * T];
                            }
                    }
                }
#pragma unroll
                for (int u = 0; u < CB; ++u) {
                    const int v = vb + u;
                    const float2 r = rho(v);
                    const float2 uu = padd(n, make_float2(-r.x, -r.y));   // n - rho (the negation folds into the add)
                    float2 m = F2(0.f);
                    if (NS == 2 || REC) m = pfma(CH2, uu, pfma(SH2, d, r));
                    if (REC && jb + v < N) {   // cells past the end of the line do not count
                        const float2 md = pfma(F2(-sh), uu, pmul(CH2, d));     // n_p' at the centre
                        const float2 ep = pfma(M1, r, m);                      // n_p - rho
                        // rc = (kappa^2, k^2 kappa^2, 1/q_s^2): registers hold q_s n_bs
                        float nb2 = 0.f;
#pragma unroll
                        for (int sp = 0; sp < NS; ++sp)
                            nb2 = fmaf(rc[2 + sp], fmaf(xn[v][sp].x, xn[v][sp].x, xn[v][sp].y * xn[v][sp].y), nb2);
                        const float e2 = fmaf(rc[0], fmaf(md.x, md.x, md.y * md.y), rc[1] * fmaf(ep.x, ep.x, ep.y * ep.y));
                        const float b2 = rc[1] * fmaf(r.x, r.x, r.y * r.y);
                        mx[0] = fmaxf(mx[0], nb2); mx[1] = fmaxf(mx[1], e2); mx[2] = fmaxf(mx[2], b2);
                    }
#pragma unroll
                    for (int sp = 0; sp < NS; ++sp) {
                        if constexpr (!UPD) continue;
                        float2 &y = xn[v][sp];
                        float2 &th = THS ? zt[THS ? u : 0][sp] : xt[THS ? 0 : v][sp];
                        float2 wv2;
                        if constexpr (UW) wv2 = W2[sp];
                        else if constexpr (THS) wv2 = F2(zw[THS ? u : 0][sp]);
                        else wv2 = sWr[(v * NS + sp) * T];
                        if (NS == 1) th = pfma(Ach, uu, pfma(Ash, d, pfma(AB, r, th)));
                        else th = pfma(F2(A[sp]), m, pfma(F2(-B[sp]), r, th));
                        y = pfma(wv2, th, y);
                        if (GM) gmax = fmaxf(gmax, fmaxf(fmaxf(fabsf(y.x), fabsf(y.y)), fmaxf(fabsf(th.x), fabsf(th.y))));
                    }
                    if constexpr (UPD) {
                        const float2 r1 = rho(v);                     // rho after the push
                        const float4 g = sG[v];
                        an = pfma(make_float2(g.x, g.y), r1, an);
                        ad = pfma(make_float2(g.z, g.w), r1, ad);
                    }
                    cross(n, d, uu, r);
                }
                if constexpr (THS && UPD) {
#pragma unroll
                    for (int u = 0; u < CB; ++u)
#pragma unroll
                        for (int sp = 0; sp < NS; ++sp) sT[((vb + u) * NS + sp) * T] = zt[u][sp];
                    // keep later batches' loads after this point: hoisting all
                    // of them would hold every cell's Theta in registers
                    asm volatile("" ::: "memory");
                }
            }
            return gmax;
        };

        // the first step's chunk aggregate (thread 0 starts from the front)
        float2 An, Ad;
        pass1(An, Ad);
        float fkm[5];        // scan scale factors (see the scan below)
        bool echg = true;    // this thread's exponent changed since fkm was formed
        // recording steps (per-mode maxima): step `it` records snapshot
        // rec_snap when it == rec_it; the one division happens here
        const bool rec_on = (a.rec_kinds & 4) != 0;
        int rec_it = -1;            // (steps of one call: int)
        long long rec_snap = 0;
        if (rec_on) {
            const long long d0 = a.step0 - a.rec_g0;   // the record clock at it = 0
            rec_snap = d0 >= 0 ? (d0 + a.rec_stride - 1) / a.rec_stride : 0;
            const long long f = rec_snap * a.rec_stride - d0;
            rec_it = f < a.n_steps ? (int)f : -1;
        }
        for (int it = 0; it < a.n_steps; ++it) {
            const float hf = (a.step0 + it) == 0 ? 0.5f : 1.0f;
            float A[NS], B[NS];
#pragma unroll
            for (int sp = 0; sp < NS; ++sp) { A[sp] = hf * Af[sp]; B[sp] = hf * Bf[sp]; }
            // ---- this step's chunk aggregate (pass 1), formed by the previous pass 2
            float2 n = An, d = Ad;
            // ---- inclusive scan over the warp's lanes
            // scale factors 2^(e_{lane - 2^k} - e), 0 for lanes below 2^k (they
            // add 0 x their own value: no divergent branch); formed again only
            // after an exponent of the warp changed (renormalisation, clamp)
            if (__any_sync(FULL, echg)) {
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const float f = p2(__shfl_up_sync(FULL, e, 1 << k) - e);
                    fkm[k] = lane >= (1 << k) ? f : 0.f;
                }
            }
            // (scalar FMAs on the shuffled components: per component the same
            // roundings as the packed form, without pairing the shuffle
            // results into register pairs)
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int dl = 1 << k;
                const float unr = __shfl_up_sync(FULL, n.x, dl), uni = __shfl_up_sync(FULL, n.y, dl);
                const float udr = __shfl_up_sync(FULL, d.x, dl), udi = __shfl_up_sync(FULL, d.y, dl);
                RotF R;
                if constexpr (THS) { const float2 r2 = sRk[k]; R = RotF{r2.x, r2.y}; } else { R = Rk[THS ? 0 : k]; }
                acc_rot(n.x, n.y, d.x, d.y, R, fkm[k], unr, uni, udr, udi);
            }
            const float fx = fkm[0];
            float2 Xn = make_float2(__fmul_rn(fx, __shfl_up_sync(FULL, n.x, 1)), __fmul_rn(fx, __shfl_up_sync(FULL, n.y, 1)));
            float2 Xd = make_float2(__fmul_rn(fx, __shfl_up_sync(FULL, d.x, 1)), __fmul_rn(fx, __shfl_up_sync(FULL, d.y, 1)));
            if (lane == 31) { sZ[buf][warp] = make_float4(n.x, n.y, d.x, d.y); sE[buf][warp] = e; }
            const int wm = __reduce_max_sync(FULL, e);
            if (lane == 0) sM[buf][warp] = wm;
            // the barrier also tells whether any exponent of the CTA changed
            // since the last clamp; if none did, every one is still in range
            const int chg = __syncthreads_or(echg ? 1 : 0);
            echg = false;
            // ---- keep within RES_SPAN of the line maximum
            if (chg) {
                int Em = RES_NONE;
                for (int ww = w0; ww < wend; ++ww) Em = max(Em, sM[buf][ww]);
                const int lo = Em - RES_SPAN;
                if (e < lo) {
                    const float f = p2(e - lo);
                    scale_chunk(f);
                    Xn = pmul(F2(f), Xn); Xd = pmul(F2(f), Xd);
                    e = lo;
                    echg = true;
                }
            }
            // ---- entry state: earlier warps of the line, then this warp's lanes
            float2 Yn = F2(0.f), Yd = F2(0.f);
            if constexpr (THS) { const float2 r2 = sRk[5]; Rw = RotF{r2.x, r2.y}; }
            for (int ww = w0; ww < warp; ++ww) {
                const float4 z = sZ[buf][ww];
                const float fz = p2(sE[buf][ww] - e);
                const float2 yn = Yn, yd = Yd;
                Yn = pmul(F2(fz), make_float2(z.x, z.y));
                Yd = pmul(F2(fz), make_float2(z.z, z.w));
                acc_rot2(Yn, Yd, Rw, 1.0f, yn, yd);
            }
            if (t == 0) {
                front_state(n, d);
            } else {
                n = Xn; d = Xd;
                if constexpr (THS) { const float2 r2 = sRl[lane]; Rl = RotF{r2.x, r2.y}; }
                acc_rot2(n, d, Rl, 1.0f, Yn, Yd);
            }
            if (a.update) An = Ad = F2(0.f);   // the next aggregate; unchanged by a field pass
            // ---- pass 2; every res_every-th step also the renormalisation
            using Y_ = std::integral_constant<bool, true>;
            using N_ = std::integral_constant<bool, false>;
            long long snap = -1;   // recording step (per-mode maxima), uniform over the CTA
            if (rec_on && it == rec_it) {
                if (rec_snap < a.rec_max_snap) snap = rec_snap;
                ++rec_snap;
                rec_it += a.rec_stride;
            }
            float gmax = 0.f;
            if (snap >= 0) {
                float mx[3] = {0.f, 0.f, 0.f};
                float rc[2 + NS];
                {
                    const int2 ix = a.items[item];
                    const int mr = min(ix.y + slot, a.M - 1);
                    const double kp = a.kap[mr], ka = a.kabs[mr];
                    rc[0] = (float)(kp * kp);
                    rc[1] = (float)(ka * ka * kp * kp);
#pragma unroll
                    for (int sp = 0; sp < NS; ++sp) {
                        const double qq = I.q[sp];
                        rc[2 + sp] = (float)(1.0 / (qq * qq));
                    }
                }
                const int e_rec = e;
                if (a.update) gmax = pass2(Y_(), Y_(), Y_(), n, d, A, B, mx, rc, An, Ad);
                else pass2(N_(), Y_(), N_(), n, d, A, B, mx, rc, An, Ad);
                // the warp's maxima at one scale 2^(2 Ew), Ew the warp's
                // largest exponent (power-of-two rescaling: exact, so the
                // maximum is that of the values; lanes more than 64 octaves
                // below it cannot hold it), reduced in FP32, then the log:
                // the mantissa part in FP32, only Ew ln 2 added in FP64 (the
                // FP64 pipe is far narrower than the FP32 one)
                const int Ew = __reduce_max_sync(FULL, has ? e_rec : RES_NONE);
                const float fsc = p2(2 * max(e_rec - Ew, -64));
                double lg[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float m = (has && mx[i] > 0.f) ? mx[i] * fsc : 0.f;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
                    lg[i] = m > 0.f ? (double)(0.5f * logf(m)) + Ew * 0.69314718055994530942 : -INFINITY;
                }
                if (lane == 0) { sMM[warp][0] = lg[0]; sMM[warp][1] = lg[1]; sMM[warp][2] = lg[2]; }
                __syncthreads();
                if (live && t == 0) {
                    double L0 = -INFINITY, L1 = -INFINITY, L2 = -INFINITY;
                    for (int ww = w0; ww < wend; ++ww) {
                        L0 = fmax(L0, sMM[ww][0]); L1 = fmax(L1, sMM[ww][1]); L2 = fmax(L2, sMM[ww][2]);
                    }
                    if (QS_CHK(a, snap * a.rec_snap_doubles + a.rec_off_mm + ((long long)itx.x + 2LL * a.n_inst) * a.Mp + mode,
                               a.rec_cap)) {
                        double *o = a.rec + snap * a.rec_snap_doubles + a.rec_off_mm + (long long)itx.x * a.Mp + mode;
                        const long long pl = (long long)a.n_inst * a.Mp;
                        o[0] = L0; o[pl] = L1; o[2 * pl] = L2;
                    }
                }
                __syncthreads();   // sMM is reused at the next recording step
            } else if ((it & (a.res_every - 1)) == a.res_every - 1) {
                gmax = pass2(Y_(), N_(), Y_(), n, d, A, B, nullptr, nullptr, An, Ad);
            } else {
                pass2(N_(), N_(), Y_(), n, d, A, B, nullptr, nullptr, An, Ad);
            }
            if (a.update) add_front(An, Ad);   // pushed rho (equilibrium front) or held value, scale e
            if (gmax > 0.f) {
                const int ex = expof(gmax);
                const int sx = clamp_shift(ex == -200 ? -126 : ex);
                if (sx > RES_HYST || sx < -RES_HYST) {
                    const float f = p2(-sx);
                    scale_chunk(f);
                    An = pmul(F2(f), An); Ad = pmul(F2(f), Ad);   // next aggregate, same scale
                    e += sx;
                    echg = true;
                }
            }
            buf ^= 1;
        }
        if (!a.update) {   // field pass: nothing to write back
            if (!a.persistent) break;
            __syncthreads();
            continue;
        }

        // write back: the threads of a 32-cell group agree on one exponent
        const long long cell0 = I.cell_off, grp0 = I.grp_off;
        int Wg = e;
#pragma unroll
        for (int o = 1; o < GRP / V; o <<= 1) Wg = max(Wg, __shfl_xor_sync(FULL, Wg, o));
        const float fo = p2(e - Wg);
        float gm = 0.f, gn = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int j = jb + v;
#pragma unroll
            for (int sp = 0; sp < NS; ++sp) {
                Cell<float> y{xn[v][sp].x, xn[v][sp].y, 0.f, 0.f};
                if constexpr (THS) {
                    const float2 z = sT[(v * NS + sp) * T];
                    y.tr = z.x; y.ti = z.y;
                } else {
                    y.tr = xt[THS ? 0 : v][sp].x; y.ti = xt[THS ? 0 : v][sp].y;
                }
                const float f = fo / q[sp];
                y.nr *= f; y.ni *= f; y.tr *= f; y.ti *= f;
                if (has && j < N) {
                    gm = fmaxf(gm, fmaxf(fmaxf(fabsf(y.nr), fabsf(y.ni)), fmaxf(fabsf(y.tr), fabsf(y.ti))));
                    gn = fmaf(y.nr + y.ti, 0.0f, gn);
                    gn = fmaf(y.ni + y.tr, 0.0f, gn);
                    st_cell(a, (cell0 + j) * NS + sp, mode, y);
                }
            }
        }
#pragma unroll
        for (int o = 1; o < GRP / V; o <<= 1) gm = fmaxf(gm, __shfl_xor_sync(FULL, gm, o));
        if (has) {
            if ((t & (GRP / V - 1)) == 0) {
                int s8 = gm > 0.0f ? expof(gm) : 0;
                s8 = s8 < -100 ? -100 : (s8 > 100 ? 100 : s8);
                const int Ws = gm > 0.0f ? Wg : 0;
                st_ex(a, grp0 + jb / GRP, mode, (Ws << 8) | (s8 & 0xff));
            }
            if (!(gn == 0.0f) || !(gm <= 3.0e38f)) atomicOr(a.err, ERR_NONFINITE);
        }
        if (!a.persistent) break;
        __syncthreads();   // shared state of this item is done before the next ticket
    }
}

// dynamic shared memory of one CTA of T threads (TT > 0: T = TT)
constexpr size_t res_smem_bytes(int NS, int V, int TT, int T) {
    return TT > 0 ? (size_t)V * NS * TT * (sizeof(float2) + sizeof(float)) : (size_t)V * NS * T * sizeof(float2);
}

}  // namespace qsk
