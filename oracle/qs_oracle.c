/*
 * qs_oracle.c -- plain, sequential FP64 CPU oracle for the linearised
 * quasistatic (QSA) beam-plasma model.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no source, header, table or helper with the
 * CUDA library: every coefficient, profile, k-grid and random number below is
 * recomputed here from its definition.
 *
 * Model (normalised units: omega_p, k_p, n_p, m_e, e; Sec. II):
 *   plasma response   (d_xi^2 + 1) n_p = rho_b = sum_s q_s n_bs       Eq. (5)
 *   pseudo-potential  (d_y^2 - 1) Psi = -n_p  ->  Psi = n_p/(1+k^2)   Eq. (14)
 *   beam continuity   d_tau n_bs = n_bs0 (d_xi v_x - d_y v_y)          Eq. (8)
 *   beam momentum     d_tau(g^3 v_x) = -(q/m) d_xi Psi,
 *                     d_tau(g v_y)   = +(q/m) d_y Psi                  Eq. (9)
 * With a transverse Fourier mode exp(i k.r_perp) and
 * Theta_s = d_xi v_x - i k.v_perp, Eqs. (8)-(9) become
 *   d_tau n_bs    = n_bs0(xi) Theta_s
 *   d_tau Theta_s = (q_s/m_s)[ (k^2/g) Psi - g^-3 d_xi^2 Psi ]
 * and with d_xi^2 Psi = kappa (rho - n_p), kappa = 1/(1+k^2) (Eqs. 5, 14):
 *   d_tau Theta_s = f1_s n_p - f2_s (rho - n_p),
 *   f1_s = (q_s/m_s) kappa k^2 / g,   f2_s = (q_s/m_s) kappa / g^3.
 * Eliminating Theta reproduces Eq. (10); dropping f2 ("reduced") gives
 * Eq. (18) for one species.
 *
 * Discretisation (the paper gives no scheme for its numerical solution of
 * Eq. (18), Sec. III.C; this is the reading the whole project uses):
 *   - xi cells j = 0..N-1 of width D, beam quantities at cell centres,
 *     rho piecewise constant on a cell.  Eq. (5) is then integrated exactly
 *     across a cell:  with P = (n_p, n_p'),
 *        P(xi + d) = R(d) P(xi) + rho (1 - cos d, sin d),
 *        R(d) = [[cos d, sin d], [-sin d, cos d]];
 *     the cell-centre value uses d = D/2, the cell exit d = D.
 *   - slow time: kick-drift leapfrog, Theta at half steps.  First step kicks
 *     by dt/2 (Theta starts at tau = 0), later steps by dt:
 *        Theta_s += h (f1_s n_mid - f2_s (rho - n_mid));
 *        n_bs    += dt n_bs0(xi_j) Theta_s.
 *   - front boundary (xi = 0): quiescent P = (0, 0); "equilibrium"
 *     P = (rho_0, 0); or a held user value per mode (Sec. III.C keeps
 *     the front value stationary).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Problem description, oracle-private.                                */
/* ------------------------------------------------------------------ */
typedef struct {
    int n_species;           /* 1 or 2                                  */
    double q[2], m[2];       /* charge (units of e), mass (units m_e)    */
    double dens[2];          /* peak n_bs0 / n_p                         */
    double gamma_b;          /* beam Lorentz factor                      */
    int reduced;             /* 1: drop the g^-3 d_xi^2 term (Eq. 18)    */
    int front;               /* 0 quiescent, 1 equilibrium, 2 held       */
    int n_xi;                /* xi cells                                 */
    double dxi, dt;          /* cell width, slow-time step               */
    const double *shape;     /* [n_xi] profile n_b0(xi_j)/peak           */
    int n_modes;
    const double *kperp2;    /* [n_modes] |k_perp|^2                     */
    const double *held;      /* [n_modes*4]: re n, im n, re n', im n'    */
} or_cfg;

/* ------------------------------------------------------------------ */
/* Longitudinal profiles n_b0(xi)/peak at cell centres xi_j=(j+1/2)D.  */
/* Flat-top with a sharp front (Sec. II/III.A), Gaussian (Sec. III.C), */
/* linear front ramp then flat top (Sec. IV.B).                        */
/* ------------------------------------------------------------------ */
int or_profile(int kind, int n_xi, double dxi, double length, double sigma,
               double center, double ramp, double *out)
{
    for (int j = 0; j < n_xi; ++j) {
        double xi = (j + 0.5) * dxi;
        double v;
        switch (kind) {
        case 0: v = (xi <= length) ? 1.0 : 0.0; break;
        case 1: { double u = (xi - center) / sigma; v = exp(-0.5 * u * u); } break;
        case 2:
            if (xi > length) v = 0.0;
            else if (ramp > 0.0 && xi < ramp) v = xi / ramp;
            else v = 1.0;
            break;
        default: return -1;
        }
        out[j] = v;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Transverse wavenumber sets.                                         */
/* 2D slab: explicit list.  3D: cell-centred n x n grid,               */
/*   k_i = (i - (n-1)/2) * 2 kmax / n,  optional disc |k| <= kmax.     */
/* Active modes are listed row-major (ix outer, iy inner).             */
/* out_idx receives the grid linear index ix*nky+iy of every active    */
/* mode, out_k2 its |k|^2, out_kabs its |k|.  Returns the count.       */
/* ------------------------------------------------------------------ */
int or_kgrid2(int nkx, int nky, double kmax, int disc, int32_t *out_idx,
              double *out_k2, double *out_kx, double *out_ky)
{
    int n = 0;
    double dkx = 2.0 * kmax / nkx, dky = 2.0 * kmax / nky;
    double lim = kmax * kmax;
    for (int ix = 0; ix < nkx; ++ix) {
        double kx = (ix - 0.5 * (nkx - 1)) * dkx;
        for (int iy = 0; iy < nky; ++iy) {
            double ky = (iy - 0.5 * (nky - 1)) * dky;
            double k2 = kx * kx + ky * ky;
            if (disc && !(k2 <= lim)) continue;
            if (out_idx) out_idx[n] = ix * nky + iy;
            if (out_k2) out_k2[n] = k2;
            if (out_kx) out_kx[n] = kx;
            if (out_ky) out_ky[n] = ky;
            ++n;
        }
    }
    return n;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator, from its published           */
/* definition (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two  */
/* 32x32->64 multiplies with the key bumped by the Weyl constants.     */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (r < 9) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two independent standard normals for counter (a,b,c,d): two 53-bit  */
/* uniforms in (0,1) from the four words, then Box-Muller.             */
static void or_normal2(uint64_t seed, uint32_t a, uint32_t b, uint32_t c,
                       uint32_t d, double *g1, double *g2)
{
    uint32_t ctr[4] = {a, b, c, d};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    uint64_t m1 = ((uint64_t)x[0] << 21) | (x[1] >> 11);
    uint64_t m2 = ((uint64_t)x[2] << 21) | (x[3] >> 11);
    double u1 = ((double)m1 + 0.5) * 0x1.0p-53;
    double u2 = ((double)m2 + 0.5) * 0x1.0p-53;
    double r = sqrt(-2.0 * log(u1));
    double th = 2.0 * M_PI * u2;
    *g1 = r * cos(th);
    *g2 = r * sin(th);
}

/* White-noise seed of the beam density (reading: complex Gaussian with
 * E|dn_b|^2 = (A*shape_j)^2 in units of n_p, Theta = 0).  Counter words:
 * (cell j, canonical mode id, instance, species).  A mode whose partner
 * -k has the smaller id receives the complex conjugate, so that the
 * perturbation is a real field in configuration space.
 * nb layout: [mode][species][j][re,im].                              */
void or_seed_noise(uint64_t seed, double amplitude, int inst, int n_modes,
                   int n_species, int n_xi, const int32_t *mode_id,
                   const int32_t *partner_id, const double *shape,
                   double *nb, double *th)
{
    const double inv_sqrt2 = 0.70710678118654752440;
    for (int mo = 0; mo < n_modes; ++mo) {
        int32_t id = mode_id[mo];
        int32_t pid = partner_id ? partner_id[mo] : id;
        int conj = pid < id;
        uint32_t cid = (uint32_t)(conj ? pid : id);
        for (int s = 0; s < n_species; ++s) {
            for (int j = 0; j < n_xi; ++j) {
                double g1, g2;
                or_normal2(seed, (uint32_t)j, cid, (uint32_t)inst, (uint32_t)s,
                           &g1, &g2);
                double a = amplitude * shape[j] * inv_sqrt2;
                size_t o = (((size_t)mo * n_species + s) * n_xi + j) * 2;
                nb[o] = a * g1;
                nb[o + 1] = conj ? -a * g2 : a * g2;
                th[o] = 0.0;
                th[o + 1] = 0.0;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* The sweep.  One call advances every mode line by n_steps slow-time  */
/* steps; `step0` is the global index of the first one (step 0 kicks   */
/* by dt/2).  Optional record of the fields at tau = (step0+i) dt for  */
/* local steps i with i % rec_stride == 0:                            */
/*   rec_mag [snap][5][mode][j]: |dn_b|, |dE|, |dB|, |F_perp|, |E_x|   */
/*   rec_np  [snap][mode][j][2]: n_p at the cell centre (complex).     */
/* Field formulas (a reading; the paper does not derive E or B, it     */
/* only states F_perp ~ grad_perp Psi, Sec. III.C): Coulomb gauge      */
/* with d_t -> d_xi, d_x -> -d_xi gives                                */
/*   E_x = -d_xi Psi,  E_perp = i k kappa (n_p - rho),                 */
/*   B_perp magnitude |k| kappa |rho|,  F_perp = E_perp - (x x B) =    */
/*   i k Psi.                                                          */
/* ------------------------------------------------------------------ */
/* Complex field components at a cell centre, each the coefficient along
 * its transverse unit vector (2D slab: E_y, B_z, F_y), from the centre
 * values n = n_p, d = n_p' and the cell's beam charge rho:
 *   v[0..1] E_x    = -kappa d                        (E_x = -d_xi Psi)
 *   v[2..3] E_perp = i |k| kappa (n - rho)
 *   v[4..5] B      = -i |k| kappa rho                 (B_z in the slab)
 *   v[6..7] F_perp = i |k| kappa n                     (= i k Psi, which
 *                    equals E_perp - B: the force on a beam particle)    */
static void field_vec(double kabs, double kap, double npr, double npi,
                      double dpr, double dpi, double rr, double ri, double *v)
{
    double a = kabs * kap;
    v[0] = -kap * dpr;           v[1] = -kap * dpi;
    v[2] = -a * (npi - ri);      v[3] = a * (npr - rr);
    v[4] = a * ri;               v[5] = -a * rr;
    v[6] = -a * npi;             v[7] = a * npr;
}

static void field_mags(double kabs, double kap, double npr, double npi,
                       double dpr, double dpi, double rr, double ri,
                       double *E, double *B, double *F, double *Ex)
{
    double v[8];
    field_vec(kabs, kap, npr, npi, dpr, dpi, rr, ri, v);
    double ex2 = v[0] * v[0] + v[1] * v[1];
    *E = sqrt(ex2 + v[2] * v[2] + v[3] * v[3]);
    *B = sqrt(v[4] * v[4] + v[5] * v[5]);
    *F = sqrt(v[6] * v[6] + v[7] * v[7]);
    *Ex = sqrt(ex2);
}

int or_sweep(const or_cfg *cfg, double *nb, double *th, long step0,
             int n_steps, int rec_stride, double *rec_mag, double *rec_np)
{
    const int N = cfg->n_xi, S = cfg->n_species, M = cfg->n_modes;
    if (N < 1 || S < 1 || S > 2 || M < 1 || cfg->dxi <= 0.0 || cfg->dt <= 0.0)
        return -1;
    if (rec_stride < 1) rec_stride = 1;
    const double D = cfg->dxi, c = cos(D), s = sin(D);
    const double ch = cos(0.5 * D), sh = sin(0.5 * D);
    const double g = cfg->gamma_b;
    const int nsnap = (n_steps + rec_stride - 1) / rec_stride;

#pragma omp parallel for schedule(dynamic, 1)
    for (int mo = 0; mo < M; ++mo) {
        const double k2 = cfg->kperp2[mo];
        const double kap = 1.0 / (1.0 + k2);
        const double kabs = sqrt(k2);
        double f1[2], f2[2];
        for (int sp = 0; sp < S; ++sp) {
            double qm = cfg->q[sp] / cfg->m[sp];
            f1[sp] = qm * kap * k2 / g;
            f2[sp] = cfg->reduced ? 0.0 : qm * kap / (g * g * g);
        }
        for (int it = 0; it < n_steps; ++it) {
            const long gstep = step0 + it;
            const double h = (gstep == 0) ? 0.5 * cfg->dt : cfg->dt;
            const int rec = (rec_mag || rec_np) && (it % rec_stride == 0);
            const int snap = it / rec_stride;
            /* front boundary value P_0 = (n, n') at xi = 0 */
            double nr = 0, ni = 0, dr = 0, di = 0;
            if (cfg->front == 1) {
                for (int sp = 0; sp < S; ++sp) {
                    size_t o = (((size_t)mo * S + sp) * N + 0) * 2;
                    nr += cfg->q[sp] * nb[o];
                    ni += cfg->q[sp] * nb[o + 1];
                }
            } else if (cfg->front == 2 && cfg->held) {
                nr = cfg->held[4 * mo + 0]; ni = cfg->held[4 * mo + 1];
                dr = cfg->held[4 * mo + 2]; di = cfg->held[4 * mo + 3];
            }
            for (int j = 0; j < N; ++j) {
                /* rho_j = sum_s q_s n_bs,j at time tau_n (before the drift) */
                double rr = 0, ri = 0;
                for (int sp = 0; sp < S; ++sp) {
                    size_t o = (((size_t)mo * S + sp) * N + j) * 2;
                    rr += cfg->q[sp] * nb[o];
                    ri += cfg->q[sp] * nb[o + 1];
                }
                /* half-cell propagation to the cell centre (Eq. 5 exact) */
                double mr = ch * nr + sh * dr + rr * (1.0 - ch);
                double mi = ch * ni + sh * di + ri * (1.0 - ch);
                double mdr = -sh * nr + ch * dr + rr * sh;
                double mdi = -sh * ni + ch * di + ri * sh;
                if (rec) {
                    double nbm2 = 0;
                    for (int sp = 0; sp < S; ++sp) {
                        size_t o = (((size_t)mo * S + sp) * N + j) * 2;
                        nbm2 += nb[o] * nb[o] + nb[o + 1] * nb[o + 1];
                    }
                    if (rec_mag) {
                        double E, B, F, Ex;
                        field_mags(kabs, kap, mr, mi, mdr, mdi, rr, ri, &E, &B, &F, &Ex);
                        size_t plane = (size_t)M * N;
                        size_t base = (size_t)snap * 5 * plane + (size_t)mo * N + j;
                        rec_mag[base + 0 * plane] = sqrt(nbm2);
                        rec_mag[base + 1 * plane] = E;
                        rec_mag[base + 2 * plane] = B;
                        rec_mag[base + 3 * plane] = F;
                        rec_mag[base + 4 * plane] = Ex;
                    }
                    if (rec_np) {
                        size_t o = (((size_t)snap * M + mo) * N + j) * 2;
                        rec_np[o] = mr;
                        rec_np[o + 1] = mi;
                    }
                }
                /* full-cell propagation to the cell exit (Eq. 5 exact) */
                double xr = c * nr + s * dr + rr * (1.0 - c);
                double xi = c * ni + s * di + ri * (1.0 - c);
                double yr = -s * nr + c * dr + rr * s;
                double yi = -s * ni + c * di + ri * s;
                nr = xr; ni = xi; dr = yr; di = yi;
                /* beam push: Eqs. (8)-(9) per mode, leapfrog in tau */
                for (int sp = 0; sp < S; ++sp) {
                    size_t o = (((size_t)mo * S + sp) * N + j) * 2;
                    double Fr = f1[sp] * mr - f2[sp] * (rr - mr);
                    double Fi = f1[sp] * mi - f2[sp] * (ri - mi);
                    th[o] += h * Fr;
                    th[o + 1] += h * Fi;
                    double n0 = cfg->dens[sp] * cfg->shape[j];
                    nb[o] += cfg->dt * n0 * th[o];
                    nb[o + 1] += cfg->dt * n0 * th[o + 1];
                }
            }
        }
    }
    (void)nsnap;
    return 0;
}

/* Field-only pass at the current state (no update), same outputs as    */
/* one snapshot of or_sweep's record.                                   */
int or_fields(const or_cfg *cfg, const double *nb, double *rec_mag, double *rec_np)
{
    const int N = cfg->n_xi, S = cfg->n_species, M = cfg->n_modes;
    size_t sz = (size_t)M * S * N * 2;
    double *nb2 = (double *)malloc(sz * sizeof(double));
    double *th2 = (double *)calloc(sz, sizeof(double));
    if (!nb2 || !th2) { free(nb2); free(th2); return -2; }
    memcpy(nb2, nb, sz * sizeof(double));
    /* one recorded step on a scratch copy; the update is discarded */
    int rc = or_sweep(cfg, nb2, th2, 1, 1, 1, rec_mag, rec_np);
    free(nb2); free(th2);
    return rc;
}

/* Zeroth-order wake: response n_p^(0) of the plasma to the unperturbed
 * beam charge rho_b0(xi_j) = sum_s q_s dens_s shape_j (Eq. 5 applied to
 * the equilibrium).  out_edge[j] = n_p at xi = (j+1) D,
 * out_mid[j] = n_p at the cell centre.                                 */
int or_wake0(const or_cfg *cfg, double *out_edge, double *out_mid)
{
    const int N = cfg->n_xi;
    const double D = cfg->dxi, c = cos(D), s = sin(D);
    const double ch = cos(0.5 * D), sh = sin(0.5 * D);
    double n = 0, d = 0;
    for (int j = 0; j < N; ++j) {
        double r = 0;
        for (int sp = 0; sp < cfg->n_species; ++sp)
            r += cfg->q[sp] * cfg->dens[sp] * cfg->shape[j];
        if (out_mid) out_mid[j] = ch * n + sh * d + r * (1.0 - ch);
        double x = c * n + s * d + r * (1.0 - c);
        double y = -s * n + c * d + r * s;
        n = x; d = y;
        if (out_edge) out_edge[j] = n;
    }
    return 0;
}

/* Complex field components at the current state (no update), for the
 * Maxwell-law pins of the field reading: out [mode][j][10] = E_x, E_perp,
 * B, F_perp (as in field_vec) and rho, each (re, im) at the cell centre,
 * with n_p at the centre from the same exact half-cell propagation.     */
int or_fields_vec(const or_cfg *cfg, const double *nb, double *out)
{
    const int N = cfg->n_xi, S = cfg->n_species, M = cfg->n_modes;
    const double D = cfg->dxi, c = cos(D), s = sin(D);
    const double ch = cos(0.5 * D), sh = sin(0.5 * D);
    for (int mo = 0; mo < M; ++mo) {
        const double k2 = cfg->kperp2[mo];
        const double kap = 1.0 / (1.0 + k2), kabs = sqrt(k2);
        double nr = 0, ni = 0, dr = 0, di = 0;
        if (cfg->front == 1) {
            for (int sp = 0; sp < S; ++sp) {
                size_t o = (((size_t)mo * S + sp) * N + 0) * 2;
                nr += cfg->q[sp] * nb[o];
                ni += cfg->q[sp] * nb[o + 1];
            }
        } else if (cfg->front == 2 && cfg->held) {
            nr = cfg->held[4 * mo + 0]; ni = cfg->held[4 * mo + 1];
            dr = cfg->held[4 * mo + 2]; di = cfg->held[4 * mo + 3];
        }
        for (int j = 0; j < N; ++j) {
            double rr = 0, ri = 0;
            for (int sp = 0; sp < S; ++sp) {
                size_t o = (((size_t)mo * S + sp) * N + j) * 2;
                rr += cfg->q[sp] * nb[o];
                ri += cfg->q[sp] * nb[o + 1];
            }
            double mr = ch * nr + sh * dr + rr * (1.0 - ch);
            double mi = ch * ni + sh * di + ri * (1.0 - ch);
            double mdr = -sh * nr + ch * dr + rr * sh;
            double mdi = -sh * ni + ch * di + ri * sh;
            double *v = out + ((size_t)mo * N + j) * 10;
            field_vec(kabs, kap, mr, mi, mdr, mdi, rr, ri, v);
            v[8] = rr; v[9] = ri;
            double xr = c * nr + s * dr + rr * (1.0 - c);
            double xi = c * ni + s * di + ri * (1.0 - c);
            double yr = -s * nr + c * dr + rr * s;
            double yi = -s * ni + c * di + ri * s;
            nr = xr; ni = xi; dr = yr; di = yi;
        }
    }
    return 0;
}

/* Threads an OpenMP parallel region of this library uses (for reporting
 * the core count of a timed oracle run). */
int or_threads(void) { return omp_get_max_threads(); }
