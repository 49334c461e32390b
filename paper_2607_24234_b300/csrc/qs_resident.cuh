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
// powers of two.  A thread renormalises its chunk when the largest mantissa
// leaves [2^-16, 2^16], and no exponent of a line may lie more than
// RES_SPAN below the line's largest (checked every step), so no scale factor
// in the scan exceeds about 2^(RES_SPAN + 17) and nothing overflows.  Only
// values below ~2^-(RES_SPAN + 126) of the line maximum flush to zero.
// On the way out the threads sharing a 32-cell group agree on one exponent
// and write the usual (mantissa, exponent word) layout.
#pragma once
#include <type_traits>

namespace qsk {

constexpr int RES_MAX_WARPS = 16;   // T <= 512
constexpr int RES_SPAN = 96;
constexpr int RES_HYST = 16;
constexpr int RES_NONE = -(1 << 20);   // exponent of a thread that holds no value yet

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
__device__ __forceinline__ int clamp_shift(int s) { return s < -126 ? -126 : (s > 126 ? 126 : s); }
// 2^e for e in [-126, 127]; 0 below (branch free)
__device__ __forceinline__ float p2(int e) { return __int_as_float((max(-127, min(e, 127)) + 127) << 23); }

template <int NS, int V>
__global__ void __launch_bounds__(512) k_sweep_res(const SweepArgs a) {
    static_assert(GRP % V == 0, "a thread's cells lie in one exponent group");
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ float sW[];             // dt n_bs0 per cell: [v * NS + sp][thread]
    __shared__ float4 sZ[2][RES_MAX_WARPS];   // inclusive warp aggregate (lane 31)
    __shared__ int sE[2][RES_MAX_WARPS];      // its exponent
    __shared__ int sM[2][RES_MAX_WARPS];      // largest exponent in the warp
    __shared__ int s_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = blockDim.x, nw = T >> 5;
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
        const InstDev I = a.inst[itx.x];
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
        const bool full = live && jb + V <= N;         // no cell of the chunk past the end
        const bool front1 = a.front == 1 && live && t == 0;

        // per-line constants
        const double kapd = a.kap[mc], kk2d = a.kapk2[mc];
        float Af[NS], Bf[NS], q[NS];
#pragma unroll
        for (int sp = 0; sp < NS; ++sp) {
            const double f1 = I.qm_g[sp] * kk2d, f2 = I.qm_g3[sp] * kapd;
            Af[sp] = (float)(I.dt * (f1 + f2));
            Bf[sp] = (float)(I.dt * f2);
            q[sp] = (float)I.q[sp];
        }
        const float c = (float)I.c, s = (float)I.s, ch = (float)I.ch, sh = (float)I.sh;
        RotF Rk[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) Rk[k] = rotf(I.dxi * (double)(V << k));
        const RotF Rl = rotf(I.dxi * (double)(V * lane));
        const RotF Rw = rotf(I.dxi * (double)(32 * V));
        const bool held = a.front == 2 && a.held != nullptr && live && t == 0;
        const double *hp = held ? a.held + ((long long)itx.x * a.Mp + mc) * 4 : nullptr;

        // load the chunk: mantissas relative to e = W + s8 of its group
        Cell<float> x[V][NS];
        int e = RES_NONE;
        float fin = 1.0f;
        if (has) {
            const int exw = __ldcg(a.ex + (I.grp_off + jb / GRP) * a.Mp + mode);
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
                if (has && j < N) {
                    const long long row = (I.cell_off + j) * NS + sp;
                    ld_cell(a, row, mode, x[v][sp]);
                    x[v][sp].nr *= fin; x[v][sp].ni *= fin; x[v][sp].tr *= fin; x[v][sp].ti *= fin;
                    wv = __ldg(reinterpret_cast<const float *>(a.w) + row);
                } else {
                    x[v][sp] = Cell<float>{0.f, 0.f, 0.f, 0.f};
                }
                sW[(v * NS + sp) * T + tid] = wv;    // only this thread reads it back
            }
        }
        auto scale_chunk = [&](float f) {
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
                for (int sp = 0; sp < NS; ++sp) {
                    x[v][sp].nr *= f; x[v][sp].ni *= f; x[v][sp].tr *= f; x[v][sp].ti *= f;
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
        auto rho = [&](int v, float &rr, float &ri) {
            rr = q[0] * x[v][0].nr; ri = q[0] * x[v][0].ni;
            if (NS == 2) { rr = fmaf(q[NS - 1], x[v][NS - 1].nr, rr); ri = fmaf(q[NS - 1], x[v][NS - 1].ni, ri); }
        };
        // front: P entering cell 0 (thread 0 of the line), in this thread's scale
        auto front_state = [&](float &nr, float &ni, float &dr, float &di) {
            nr = ni = dr = di = 0.f;
            if (held) {
                nr = (float)ldexp(hp[0], -e); ni = (float)ldexp(hp[1], -e);
                dr = (float)ldexp(hp[2], -e); di = (float)ldexp(hp[3], -e);
            }
            if (front1) rho(0, nr, ni);   // equilibrium front: n_p = rho, n_p' = 0 at xi = 0
        };
        // pass 1: the chunk's response from the given entry state
        auto pass1 = [&](auto chk, float &nr, float &ni, float &dr, float &di) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (decltype(chk)::value && jb + v >= N) break;
                float rr, ri;
                rho(v, rr, ri);
                const float ur = nr - rr, ui = ni - ri;
                const float xr = fmaf(c, ur, fmaf(s, dr, rr)), xi = fmaf(c, ui, fmaf(s, di, ri));
                dr = fmaf(-s, ur, c * dr);
                di = fmaf(-s, ui, c * di);
                nr = xr; ni = xi;
            }
        };
        // pass 2: fields at the cell centre and the push
        auto pass2 = [&](auto chk, float nr, float ni, float dr, float di, const float *A, const float *B) {
            float gmax = 0.f;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (decltype(chk)::value && jb + v >= N) break;
                float rr, ri;
                rho(v, rr, ri);
                const float ur = nr - rr, ui = ni - ri;
                const float mr = fmaf(ch, ur, fmaf(sh, dr, rr)), mi = fmaf(ch, ui, fmaf(sh, di, ri));
                const float xr = fmaf(c, ur, fmaf(s, dr, rr)), xi = fmaf(c, ui, fmaf(s, di, ri));
                dr = fmaf(-s, ur, c * dr);
                di = fmaf(-s, ui, c * di);
                nr = xr; ni = xi;
#pragma unroll
                for (int sp = 0; sp < NS; ++sp) {
                    Cell<float> &y = x[v][sp];
                    const float wv = sW[(v * NS + sp) * T + tid];
                    y.tr = fmaf(A[sp], mr, fmaf(-B[sp], rr, y.tr));
                    y.ti = fmaf(A[sp], mi, fmaf(-B[sp], ri, y.ti));
                    y.nr = fmaf(wv, y.tr, y.nr);
                    y.ni = fmaf(wv, y.ti, y.ni);
                    gmax = fmaxf(gmax, fmaxf(fmaxf(fabsf(y.nr), fabsf(y.ni)), fmaxf(fabsf(y.tr), fabsf(y.ti))));
                }
            }
            return gmax;
        };
        using Yes = std::integral_constant<bool, true>;
        using No = std::integral_constant<bool, false>;

        for (int it = 0; it < a.n_steps; ++it) {
            const float hf = (a.step0 + it) == 0 ? 0.5f : 1.0f;
            float A[NS], B[NS];
#pragma unroll
            for (int sp = 0; sp < NS; ++sp) { A[sp] = hf * Af[sp]; B[sp] = hf * Bf[sp]; }
            // ---- pass 1 (thread 0 starts from the front, the others from 0)
            float nr, ni, dr, di;
            front_state(nr, ni, dr, di);
            if (full) pass1(No(), nr, ni, dr, di);
            else if (has) pass1(Yes(), nr, ni, dr, di);
            // ---- inclusive scan over the warp's lanes
            float fk[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) fk[k] = p2(__shfl_up_sync(FULL, e, 1 << k) - e);
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int d = 1 << k;
                const float ur = __shfl_up_sync(FULL, nr, d), ui = __shfl_up_sync(FULL, ni, d);
                const float vr = __shfl_up_sync(FULL, dr, d), vi = __shfl_up_sync(FULL, di, d);
                if (lane >= d) acc_rot(nr, ni, dr, di, Rk[k], fk[k], ur, ui, vr, vi);
            }
            float Xr = __shfl_up_sync(FULL, nr, 1), Xi = __shfl_up_sync(FULL, ni, 1);
            float Xdr = __shfl_up_sync(FULL, dr, 1), Xdi = __shfl_up_sync(FULL, di, 1);
            const float fx = lane == 0 ? 0.f : fk[0];
            Xr *= fx; Xi *= fx; Xdr *= fx; Xdi *= fx;
            if (lane == 31) { sZ[buf][warp] = make_float4(nr, ni, dr, di); sE[buf][warp] = e; }
            const int wm = __reduce_max_sync(FULL, e);
            if (lane == 0) sM[buf][warp] = wm;
            __syncthreads();
            // ---- keep within RES_SPAN of the line maximum
            {
                int Em = RES_NONE;
                for (int ww = w0; ww < wend; ++ww) Em = max(Em, sM[buf][ww]);
                const int lo = Em - RES_SPAN;
                if (e < lo) {
                    const float f = p2(e - lo);
                    scale_chunk(f);
                    Xr *= f; Xi *= f; Xdr *= f; Xdi *= f;
                    e = lo;
                }
            }
            // ---- entry state: earlier warps of the line, then this warp's lanes
            float Yr = 0.f, Yi = 0.f, Ydr = 0.f, Ydi = 0.f;
            for (int ww = w0; ww < warp; ++ww) {
                const float4 z = sZ[buf][ww];
                const float fz = p2(sE[buf][ww] - e);
                const float yr = fmaf(Rw.c, Yr, Rw.s * Ydr), yi = fmaf(Rw.c, Yi, Rw.s * Ydi);
                const float ydr = fmaf(-Rw.s, Yr, Rw.c * Ydr), ydi = fmaf(-Rw.s, Yi, Rw.c * Ydi);
                Yr = fmaf(fz, z.x, yr); Yi = fmaf(fz, z.y, yi);
                Ydr = fmaf(fz, z.z, ydr); Ydi = fmaf(fz, z.w, ydi);
            }
            if (t == 0) {
                front_state(nr, ni, dr, di);
            } else {
                nr = Xr; ni = Xi; dr = Xdr; di = Xdi;
                acc_rot(nr, ni, dr, di, Rl, 1.0f, Yr, Yi, Ydr, Ydi);
            }
            // ---- pass 2
            float gmax = 0.f;
            if (full) gmax = pass2(No(), nr, ni, dr, di, A, B);
            else if (has) gmax = pass2(Yes(), nr, ni, dr, di, A, B);
            // ---- own renormalisation (hysteresis)
            if (gmax > 0.f) {
                const int ex = expof(gmax);
                const int sx = clamp_shift(ex == -200 ? -126 : ex);
                if (sx > RES_HYST || sx < -RES_HYST) { scale_chunk(p2(-sx)); e += sx; }
            }
            buf ^= 1;
        }

        // write back: the threads of a 32-cell group agree on one exponent
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
                Cell<float> &y = x[v][sp];
                y.nr *= fo; y.ni *= fo; y.tr *= fo; y.ti *= fo;
                if (has && j < N) {
                    gm = fmaxf(gm, fmaxf(fmaxf(fabsf(y.nr), fabsf(y.ni)), fmaxf(fabsf(y.tr), fabsf(y.ti))));
                    gn = fmaf(y.nr + y.ti, 0.0f, gn);
                    gn = fmaf(y.ni + y.tr, 0.0f, gn);
                    st_cell(a, (I.cell_off + j) * NS + sp, mode, y);
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
                __stcg(a.ex + (I.grp_off + jb / GRP) * a.Mp + mode, (Ws << 8) | (s8 & 0xff));
            }
            if (!(gn == 0.0f) || !(gm <= 3.0e38f)) atomicOr(a.err, ERR_NONFINITE);
        }
        if (!a.persistent) break;
        __syncthreads();   // shared state of this item is done before the next ticket
    }
}

}  // namespace qsk
