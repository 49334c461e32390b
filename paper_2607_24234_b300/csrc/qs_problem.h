// qs_problem.h -- host-side reading of a qs_params problem statement,
// shared by every entry point that takes one (qs_init, qs_sweep_noalloc).
//
// Sec. II states the problem as beam species (q_s, m_s, n_bs0), gamma_b, a
// longitudinal profile, the transverse wavenumbers and the xi / tau grids;
// these helpers check such a statement, evaluate the profile at the cell
// centres and list the active transverse modes.  Header-only, host code.
#pragma once

#include <cmath>
#include <cstdio>
#include <vector>

#include "qs.h"

namespace qsp {

// Check one problem statement.  On failure returns the status and writes a
// message (instance index `idx`) to msg.
inline qs_status validate(const qs_params &p, int idx, char *msg, size_t msg_len) {
#define QSP_BAD(st, ...)                         \
    do {                                         \
        snprintf(msg, msg_len, __VA_ARGS__);     \
        return (st);                             \
    } while (0)
    if (p.geom != QS_GEOM_KLIST && p.geom != QS_GEOM_KGRID2)
        QSP_BAD(p.geom == 2 ? QS_ERR_UNSUPPORTED : QS_ERR_ARG, "instance %d: geom %d", idx, p.geom);
    if (p.prec != QS_FP64 && p.prec != QS_FP32_RENORM) QSP_BAD(QS_ERR_ARG, "instance %d: prec", idx);
    if (p.model != QS_MODEL_FULL && p.model != QS_MODEL_REDUCED) QSP_BAD(QS_ERR_ARG, "instance %d: model", idx);
    if (p.front < 0 || p.front > 2) QSP_BAD(QS_ERR_ARG, "instance %d: front", idx);
    if (p.n_species < 1 || p.n_species > 2) QSP_BAD(QS_ERR_ARG, "instance %d: n_species must be 1 or 2", idx);
    for (int s = 0; s < p.n_species; ++s) {
        const qs_species &sp = p.species[s];
        if (!(sp.m > 0.0) || !(sp.density_ratio >= 0.0) || !std::isfinite(sp.q) || !std::isfinite(sp.m) ||
            !std::isfinite(sp.density_ratio))
            QSP_BAD(QS_ERR_ARG, "instance %d: species %d needs finite q, m > 0, density >= 0", idx, s);
    }
    if (!(p.gamma_b > 1.0) || !std::isfinite(p.gamma_b)) QSP_BAD(QS_ERR_ARG, "instance %d: gamma_b must be > 1", idx);
    if (p.n_xi < 1) QSP_BAD(QS_ERR_ARG, "instance %d: n_xi must be >= 1", idx);
    if (!(p.dxi > 0.0) || !std::isfinite(p.dxi)) QSP_BAD(QS_ERR_ARG, "instance %d: dxi must be > 0", idx);
    if (!(p.dt > 0.0) || !std::isfinite(p.dt)) QSP_BAD(QS_ERR_ARG, "instance %d: dt must be > 0", idx);
    if (p.profile < 0 || p.profile > 3) QSP_BAD(QS_ERR_ARG, "instance %d: profile", idx);
    if (p.profile == QS_PROF_GAUSSIAN && !(p.sigma_xi > 0.0 && std::isfinite(p.sigma_xi)))
        QSP_BAD(QS_ERR_ARG, "instance %d: sigma_xi", idx);
    if (p.profile == QS_PROF_USER && !p.user_profile) QSP_BAD(QS_ERR_ARG, "instance %d: user_profile", idx);
    if (p.geom == QS_GEOM_KLIST && (p.n_k < 1 || !p.k_list)) QSP_BAD(QS_ERR_ARG, "instance %d: k_list", idx);
    if (p.geom == QS_GEOM_KLIST)
        for (int i = 0; i < p.n_k; ++i)
            if (!std::isfinite(p.k_list[i])) QSP_BAD(QS_ERR_ARG, "instance %d: k_list[%d] is not finite", idx, i);
    if (p.profile == QS_PROF_USER)
        for (int j = 0; j < p.n_xi; ++j)
            if (!std::isfinite(p.user_profile[j]))
                QSP_BAD(QS_ERR_ARG, "instance %d: user_profile[%d] is not finite", idx, j);
    if (p.geom == QS_GEOM_KGRID2 && (p.nkx < 1 || p.nky < 1 || !(p.kmax > 0.0) || !std::isfinite(p.kmax)))
        QSP_BAD(QS_ERR_ARG, "instance %d: kgrid", idx);
    if (p.front == QS_FRONT_HELD && !p.held_front) QSP_BAD(QS_ERR_ARG, "instance %d: held_front", idx);
    return QS_OK;
#undef QSP_BAD
}

// Longitudinal profile n_b0(xi_j)/peak at the cell centres xi_j = (j + 1/2)
// dxi: flat top with a sharp front (Sec. III.A), Gaussian (Sec. III.C),
// linear front ramp then flat top (Sec. IV.B), or the caller's values.
inline bool profile_shape(const qs_params &p, std::vector<double> &out) {
    out.resize(p.n_xi);
    for (int j = 0; j < p.n_xi; ++j) {
        const double xi = (j + 0.5) * p.dxi;
        double v = 0.0;
        switch (p.profile) {
        case QS_PROF_FLATTOP: v = xi <= p.length ? 1.0 : 0.0; break;
        case QS_PROF_GAUSSIAN: {
            const double u = (xi - p.center_xi) / p.sigma_xi;
            v = std::exp(-0.5 * u * u);
        } break;
        case QS_PROF_RAMP_FLATTOP:
            v = xi > p.length ? 0.0 : (p.ramp_len > 0.0 && xi < p.ramp_len ? xi / p.ramp_len : 1.0);
            break;
        case QS_PROF_USER:
            if (!p.user_profile) return false;
            v = p.user_profile[j];
            break;
        default: return false;
        }
        out[j] = v;
    }
    return true;
}

// Active transverse modes, row-major over the grid: KLIST as given (k along
// one axis); KGRID2 the cell-centred grid k_i = (i - (n-1)/2) 2 kmax / n with
// the optional disc |k| <= kmax.  mode_id is the grid index, partner_id the
// index of -k (the mode that carries the conjugate perturbation).
struct ModeList {
    std::vector<double> kx, ky, k2;
    std::vector<int> mode_id, partner_id;
};

inline void build_modes(const qs_params &p, ModeList &m) {
    m = ModeList{};
    if (p.geom == QS_GEOM_KLIST) {
        for (int i = 0; i < p.n_k; ++i) {
            const double k = p.k_list[i];
            m.kx.push_back(k); m.ky.push_back(0.0); m.k2.push_back(k * k);
            m.mode_id.push_back(i); m.partner_id.push_back(i);
        }
        return;
    }
    const double dkx = 2.0 * p.kmax / p.nkx, dky = 2.0 * p.kmax / p.nky, lim = p.kmax * p.kmax;
    for (int ix = 0; ix < p.nkx; ++ix) {
        const double kx = (ix - 0.5 * (p.nkx - 1)) * dkx;
        for (int iy = 0; iy < p.nky; ++iy) {
            const double ky = (iy - 0.5 * (p.nky - 1)) * dky;
            const double k2 = kx * kx + ky * ky;
            if (p.disc_mask && !(k2 <= lim)) continue;
            m.kx.push_back(kx); m.ky.push_back(ky); m.k2.push_back(k2);
            m.mode_id.push_back(ix * p.nky + iy);
            m.partner_id.push_back((p.nkx - 1 - ix) * p.nky + (p.nky - 1 - iy));
        }
    }
}

// Upper bound (e-folds per slow-time step) of the growth of the scheme's
// state, in the max norm, from the problem statement alone.  One step maps
// (n_b, Theta) by Theta' = Theta + h F[n_b], n_b' = n_b + dt n_b0 Theta' with
// h <= dt, |F[n_b]| <= a |n_b| / dt and |dt n_b0| <= b, where the kick is
// (q/m)[kappa k^2 / gamma n_p - kappa / gamma^3 (rho - n_p)] (Eqs. 8-9, 14)
// with kappa k^2 <= 1, kappa <= 1, and the plasma response of Eq. (5) over a
// line of length L obeys |n_p| <= L max|rho|:
//   a = dt max_s |q_s/m_s| (1/gamma + 1/gamma^3) sum_s |q_s| (2 + L),
//   b = dt max_s n_bs0,peak max_j shape_j.
// The max norms then obey (|n_b'|, |Theta'|) <= [[1 + ab, b], [a, 1]]
// (|n_b|, |Theta|) componentwise.  In the weights (|n_b|, sqrt(b/a)
// |Theta|) that matrix is symmetric, [[1 + ab, sqrt(ab)], [sqrt(ab), 1]],
// so after k steps the weighted pair is at most rho^k times its 2-norm,
// rho = 1 + ab/2 + sqrt(ab + (ab)^2 / 4) its spectral radius: ln rho bounds
// the growth per step, and the change of weights and of norms costs a
// one-time factor sqrt(2 max(a, b) / min(a, b)) (its log in *log_cond).
// Both are 0 when a b = 0 (no coupling).
inline double growth_bound(const qs_params &p, const std::vector<double> &shape, double *log_cond) {
    double qm = 0.0, qs = 0.0, dmax = 0.0, smax = 0.0;
    for (int s = 0; s < p.n_species; ++s) {
        qm = std::max(qm, std::fabs(p.species[s].q / p.species[s].m));
        qs += std::fabs(p.species[s].q);
        dmax = std::max(dmax, p.species[s].density_ratio);
    }
    for (double v : shape) smax = std::max(smax, std::fabs(v));
    const double g = p.gamma_b, L = p.n_xi * p.dxi;
    const double a = p.dt * qm * (1.0 / g + 1.0 / (g * g * g)) * qs * (2.0 + L);
    const double b = p.dt * dmax * smax;
    const double ab = a * b;
    if (!(ab > 0.0)) {
        if (log_cond) *log_cond = 0.0;
        return 0.0;
    }
    if (log_cond) *log_cond = 0.5 * std::fabs(std::log(a / b)) + 0.5 * std::log(2.0);
    return std::log(1.0 + 0.5 * ab + std::sqrt(ab + 0.25 * ab * ab));
}

// Renormalisation interval of the resident FP32 sweep for a growth bound g
// (e-folds per step), one-time factor lc and line length L: the largest power
// of two up to 16 steps over which the state's growth stays inside the FP32
// headroom between checks.  After a check a thread's mantissas are below
// 2^16, other threads' values reach it at most 2^64 (RES_SPAN) larger, and
// the plasma partials sum at most 2 L of those, so the growth G between two
// checks must keep 2^(16 + 64) 2L G below 2^128 (half a bit to spare); 0
// when even a check every step cannot.
inline int res_every_for(double g, double lc, double L) {
    const double bits = 128.0 - 16.0 - 64.0 - std::log2(std::max(32.0, 2.0 * L)) - 0.5;
    const double budget = bits * std::log(2.0);
    for (int every = 16; every >= 1; every >>= 1)
        if (every * g + lc <= budget) return every;
    return 0;
}

}  // namespace qsp
