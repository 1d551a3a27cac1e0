// Phase-boundary extraction (§3.4 results, Table 3.1): peaks of C_V(T) and
// chi(T) on a temperature scan, refined by the three-point parabola, and the
// zero-field limit of the chi peak temperature from the least-squares fit
// T_p(hbar) = a + b hbar^c (the fit whose a, b, c the thesis prints for
// Delta = 0.32; a is the zero-field T_c of Table 3.1).
//
// hotrg_find_peaks and hotrg_fit_tc are host arithmetic on a few hundred
// scalars; hotrg_phase_scan submits its HOTRG points to the batch runner
// (hotrg_run_batch) in two batches, one per tensor kind, so every point of
// the scan runs in the library's kernels.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int FIT_GRID = 2001;
constexpr double FIT_C_LO = 0.05, FIT_C_HI = 2.0;

bool all_finite(const double* a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// Height of y[k] above the higher of its two bases (the smallest values met
// walking out from k until a strictly higher value or the end).
double prominence_at(const double* y, int n, int k) {
    double lo_l = y[k], lo_r = y[k];
    for (int i = k; i >= 0 && y[i] <= y[k]; --i) lo_l = std::min(lo_l, y[i]);
    for (int i = k; i < n && y[i] <= y[k]; ++i) lo_r = std::min(lo_r, y[i]);
    return y[k] - std::max(lo_l, lo_r);
}

// Vertex of the parabola through (x[k-1..k+1], y[k-1..k+1]) from divided
// differences, in the local coordinate u = x - x[k]: p(u) = y_k + B u + A u^2.
void parabola_vertex(const double* x, const double* y, int k, double* xv, double* yv) {
    const double w0 = x[k] - x[k - 1], w1 = x[k + 1] - x[k];
    const double d0 = (y[k] - y[k - 1]) / w0, d1 = (y[k + 1] - y[k]) / w1;
    const double A = (d1 - d0) / (w0 + w1);
    const double B = d0 + A * w0;
    if (y[k - 1] == y[k] && y[k] == y[k + 1]) {  // flat window: no vertex, the sample itself
        *xv = x[k];
        *yv = y[k];
        return;
    }
    *xv = x[k] - B / (2.0 * A);
    *yv = y[k] - B * B / (4.0 * A);
}

// Linear least squares t ~ a + b z with z_i = exp(c ln h_i), by centred sums.
struct LinFit {
    double a, b, rss, g;  // g: d rss / dc of the profile (envelope theorem)
};

LinFit lin_fit(const std::vector<double>& lh, const double* t, double c, std::vector<double>& z) {
    const int n = (int)lh.size();
    double zm = 0.0, tm = 0.0;
    for (int i = 0; i < n; ++i) {
        z[i] = std::exp(c * lh[i]);
        zm += z[i];
        tm += t[i];
    }
    zm /= n;
    tm /= n;
    double szz = 0.0, szt = 0.0;
    for (int i = 0; i < n; ++i) {
        szz += (z[i] - zm) * (z[i] - zm);
        szt += (z[i] - zm) * (t[i] - tm);
    }
    LinFit f;
    f.b = szt / szz;
    f.a = tm - f.b * zm;
    f.rss = 0.0;
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        const double r = t[i] - f.a - f.b * z[i];
        f.rss += r * r;
        s += r * z[i] * lh[i];
    }
    f.g = -2.0 * f.b * s;
    return f;
}

// Inverse of a symmetric positive definite 3 x 3 matrix (row-major) by
// Cholesky on the unit-diagonal scaling; false when it is not positive definite.
bool spd_inverse3(const double M[9], double out[9]) {
    double d[3], S[9];
    for (int i = 0; i < 3; ++i) {
        if (!(M[i * 4] > 0)) return false;
        d[i] = 1.0 / std::sqrt(M[i * 4]);
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[i * 3 + j] = M[i * 3 + j] * d[i] * d[j];
    double L[9] = {0};
    for (int j = 0; j < 3; ++j) {
        double s = S[j * 3 + j];
        for (int k = 0; k < j; ++k) s -= L[j * 3 + k] * L[j * 3 + k];
        if (!(s > 0)) return false;
        L[j * 3 + j] = std::sqrt(s);
        for (int i = j + 1; i < 3; ++i) {
            double r = S[i * 3 + j];
            for (int k = 0; k < j; ++k) r -= L[i * 3 + k] * L[j * 3 + k];
            L[i * 3 + j] = r / L[j * 3 + j];
        }
    }
    // S^-1 = L^-T L^-1: solve L X = e_c, then L^T Y = X, column by column
    for (int c = 0; c < 3; ++c) {
        double x[3], yv[3];
        for (int i = 0; i < 3; ++i) {
            double r = i == c ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) r -= L[i * 3 + k] * x[k];
            x[i] = r / L[i * 3 + i];
        }
        for (int i = 2; i >= 0; --i) {
            double r = x[i];
            for (int k = i + 1; k < 3; ++k) r -= L[k * 3 + i] * yv[k];
            yv[i] = r / L[i * 3 + i];
        }
        for (int i = 0; i < 3; ++i) out[i * 3 + c] = yv[i] * d[i] * d[c];
    }
    return true;
}

bool resolve_bracket(double c_lo, double c_hi, double* lo, double* hi) {
    if (c_lo <= 0 && c_hi <= 0) {
        *lo = FIT_C_LO;
        *hi = FIT_C_HI;
        return true;
    }
    if (!std::isfinite(c_lo) || !std::isfinite(c_hi) || !(c_lo > 0) || !(c_lo <= c_hi)) return false;
    *lo = c_lo;
    *hi = c_hi;
    return true;
}

int distinct_count(const double* v, int n) {
    std::vector<double> s(v, v + n);
    std::sort(s.begin(), s.end());
    return (int)(std::unique(s.begin(), s.end()) - s.begin());
}

void nan_fit(hotrg_tc_fit* out) {
    const double nan = std::nan("");
    out->a = out->b = out->c = nan;
    out->a_err = out->b_err = out->c_err = nan;
    out->rss = nan;
    out->n = 0;
    out->at_bound = 0;
}

}  // namespace

extern "C" {

hotrg_status hotrg_find_peaks(const double* x, const double* y, int32_t n, double min_prominence, int32_t cap,
                              double* x_peak, double* y_peak, double* prominence, int32_t* n_found) {
    if (!x || !y || !n_found || n < 0 || cap < 0 || (cap > 0 && (!x_peak || !y_peak))) return HOTRG_EINVAL;
    if (!std::isfinite(min_prominence) || !all_finite(x, n) || !all_finite(y, n)) return HOTRG_EINVAL;
    for (int i = 1; i < n; ++i)
        if (!(x[i] > x[i - 1])) return HOTRG_EINVAL;
    // runs of equal consecutive values; a run strictly above both neighbouring
    // runs (neither the first nor the last run) is a peak at its middle
    std::vector<int> rs, re;
    for (int i = 0; i < n;) {
        int j = i;
        while (j + 1 < n && y[j + 1] == y[i]) ++j;
        rs.push_back(i);
        re.push_back(j);
        i = j + 1;
    }
    struct Cand {
        int k;
        double prom;
    };
    std::vector<Cand> cand;
    for (size_t r = 1; r + 1 < rs.size(); ++r) {
        const double v = y[rs[r]];
        if (y[rs[r - 1]] < v && y[rs[r + 1]] < v) {
            const int k = (rs[r] + re[r]) / 2;
            const double p = prominence_at(y, n, k);
            if (p >= min_prominence) cand.push_back({k, p});
        }
    }
    *n_found = (int32_t)cand.size();
    std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) { return a.prom > b.prom; });
    if ((int)cand.size() > cap) cand.resize(cap);
    std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) { return a.k < b.k; });
    for (size_t i = 0; i < cand.size(); ++i) {
        parabola_vertex(x, y, cand[i].k, &x_peak[i], &y_peak[i]);
        if (prominence) prominence[i] = cand[i].prom;
    }
    return HOTRG_OK;
}

hotrg_status hotrg_fit_tc(const double* hbar, const double* t_peak, int32_t n, double c_lo, double c_hi,
                          hotrg_tc_fit* out) {
    if (!hbar || !t_peak || !out || n < 3) return HOTRG_EINVAL;
    nan_fit(out);
    double lo, hi;
    if (!resolve_bracket(c_lo, c_hi, &lo, &hi) || !all_finite(hbar, n) || !all_finite(t_peak, n))
        return HOTRG_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!(hbar[i] > 0)) return HOTRG_EINVAL;
    if (distinct_count(hbar, n) < 3) return HOTRG_EINVAL;
    std::vector<double> lh(n), z(n);
    for (int i = 0; i < n; ++i) lh[i] = std::log(hbar[i]);

    double c;
    int at_bound = 0;
    if (lo == hi) {
        c = lo;
        at_bound = 1;
    } else {
        // profile on the grid, then the stationary point around its minimum
        int kbest = 0;
        double best = INFINITY;
        std::vector<double> grid(FIT_GRID);
        for (int k = 0; k < FIT_GRID; ++k) {
            grid[k] = k == FIT_GRID - 1 ? hi : lo + (hi - lo) * k / (FIT_GRID - 1);
            const double r = lin_fit(lh, t_peak, grid[k], z).rss;
            if (r < best) {
                best = r;
                kbest = k;
            }
        }
        if (kbest == 0 && lin_fit(lh, t_peak, grid[0], z).g >= 0) {
            c = grid[0];
            at_bound = 1;
        } else if (kbest == FIT_GRID - 1 && lin_fit(lh, t_peak, grid[FIT_GRID - 1], z).g <= 0) {
            c = grid[FIT_GRID - 1];
            at_bound = 1;
        } else {
            double a = grid[std::max(kbest - 1, 0)], b = grid[std::min(kbest + 1, FIT_GRID - 1)];
            double fa = lin_fit(lh, t_peak, a, z).g, fb = lin_fit(lh, t_peak, b, z).g;
            if (fa == 0) {
                c = a;
            } else if (fb == 0) {
                c = b;
            } else if (!(fa < 0 && fb > 0)) {
                return HOTRG_ENOCONV;
            } else {
                // Illinois false position, with a bisection whenever a step
                // fails to halve the bracket; stops at the rounding level
                int side = 0;
                c = 0.5 * (a + b);
                for (int it = 0; it < 400 && b - a > 4 * DBL_EPSILON * std::max(std::fabs(a), std::fabs(b)); ++it) {
                    const double w = b - a;
                    double m = (a * fb - b * fa) / (fb - fa);
                    if (!(m > a && m < b)) m = 0.5 * (a + b);
                    const double fm = lin_fit(lh, t_peak, m, z).g;
                    c = m;
                    if (fm == 0) {
                        a = b = m;
                        break;
                    }
                    if (fm < 0) {
                        a = m;
                        fa = fm;
                        if (side == -1) fb *= 0.5;
                        side = -1;
                    } else {
                        b = m;
                        fb = fm;
                        if (side == 1) fa *= 0.5;
                        side = 1;
                    }
                    if (b - a > 0.5 * w) {
                        const double h = 0.5 * (a + b);
                        const double fh = lin_fit(lh, t_peak, h, z).g;
                        c = h;
                        if (fh == 0) {
                            a = b = h;
                            break;
                        }
                        if (fh < 0) {
                            a = h;
                            fa = fh;
                        } else {
                            b = h;
                            fb = fh;
                        }
                        side = 0;
                    }
                }
                if (b - a > 4 * DBL_EPSILON * std::max(std::fabs(a), std::fabs(b)) * 16) return HOTRG_ENOCONV;
                c = std::fabs(fa) <= std::fabs(fb) ? a : b;
            }
        }
    }
    const LinFit f = lin_fit(lh, t_peak, c, z);
    out->a = f.a;
    out->b = f.b;
    out->c = c;
    out->rss = f.rss;
    out->n = n;
    out->at_bound = at_bound;
    out->a_err = out->b_err = out->c_err = 0.0;
    if (n > 3) {
        double M[9] = {0}, Mi[9];
        for (int i = 0; i < n; ++i) {
            const double J[3] = {1.0, z[i], f.b * z[i] * lh[i]};
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s) M[r * 3 + s] += J[r] * J[s];
        }
        if (spd_inverse3(M, Mi)) {
            const double s2 = f.rss / (n - 3);
            out->a_err = std::sqrt(s2 * Mi[0]);
            out->b_err = std::sqrt(s2 * Mi[4]);
            out->c_err = std::sqrt(s2 * Mi[8]);
        } else {
            out->a_err = out->b_err = out->c_err = std::nan("");
        }
    }
    return HOTRG_OK;
}

hotrg_status hotrg_phase_scan(hotrg_ctx* ctx, const hotrg_params* base, const double* temps, int32_t n_t,
                              const double* hbar, int32_t n_h, const hotrg_phase_opts* opts, double* cv,
                              double* chi, double* t_peak, hotrg_tc_fit* fit, int32_t* field_used) {
    if (!ctx) return HOTRG_EINVAL;
    ctx->last_error.clear();
    auto bad = [ctx](const char* m) { return ::hotrg::set_err(ctx, HOTRG_EINVAL, m); };
    if (!base || !temps || !opts || n_t < 3 || n_h < 0)
        return bad("phase scan: need base, temps, opts, n_t >= 3 and n_h >= 0");
    if (n_h > 0 && (!hbar || !chi)) return bad("phase scan: hbar and chi are required when n_h > 0");
    if (base->tkind != HOTRG_T_PURE) return bad("phase scan: the gXY model only (tkind HOTRG_T_PURE)");
    for (int j = 0; j < n_t; ++j)
        if (!std::isfinite(temps[j]) || !(temps[j] > 0) || (j > 0 && !(temps[j] > temps[j - 1])))
            return bad("phase scan: temps must be finite, positive and strictly ascending");
    if (!(opts->dh > 0) || !std::isfinite(opts->dh)) return bad("phase scan: dh must be positive and finite");
    if (cv && (!(opts->hb > 0) || !std::isfinite(opts->hb))) return bad("phase scan: hb must be positive");
    for (int k = 0; k < n_h; ++k)
        if (!std::isfinite(hbar[k]) || !(hbar[k] - opts->dh >= 0))
            return bad("phase scan: every hbar must be finite and >= dh");
    if (opts->nstreams < 0 || opts->nstreams > 16) return bad("phase scan: nstreams must lie in [0, 16]");
    if (opts->field != 0 && opts->field != HOTRG_T_IMP_M && opts->field != HOTRG_T_IMP_M1)
        return bad("phase scan: field must be 0, HOTRG_T_IMP_M or HOTRG_T_IMP_M1");
    if (!std::isfinite(opts->min_prominence)) return bad("phase scan: min_prominence must be finite");
    double clo, chi_c;
    if (!resolve_bracket(opts->c_lo, opts->c_hi, &clo, &chi_c))
        return bad("phase scan: need 0 < c_lo <= c_hi (or both <= 0 for the default bracket)");
    const int kind = opts->field != 0 ? opts->field : (base->delta > 0.36 ? HOTRG_T_IMP_M : HOTRG_T_IMP_M1);
    if (field_used) *field_used = kind;
    if (fit) nan_fit(fit);

    hotrg_params q = *base;
    q.h = 0.0;
    q.h1 = 0.0;
    auto run = [&](std::vector<hotrg_params>& pp, int imp, std::vector<hotrg_result>& rr) {
        rr.assign(pp.size(), hotrg_result{});
        hotrg_status s = hotrg_run_batch(ctx, pp.data(), (int32_t)pp.size(), imp, opts->nstreams, rr.data());
        if (s != HOTRG_OK) return s;
        for (const hotrg_result& r : rr)
            if (r.status != HOTRG_OK) return (hotrg_status)r.status;
        return HOTRG_OK;
    };
    if (cv) {
        // (beta, beta + hb, beta - hb) at zero field, the order and arithmetic of hotrg_observables
        std::vector<hotrg_params> pp((size_t)3 * n_t, q);
        std::vector<hotrg_result> rr;
        for (int j = 0; j < n_t; ++j) {
            const double beta = 1.0 / temps[j];
            pp[(size_t)3 * j].beta = beta;
            pp[(size_t)3 * j + 1].beta = beta + opts->hb;
            pp[(size_t)3 * j + 2].beta = beta - opts->hb;
        }
        hotrg_status s = run(pp, HOTRG_T_PURE, rr);
        if (s != HOTRG_OK) return s;
        for (int j = 0; j < n_t; ++j) {
            const double beta = 1.0 / temps[j];
            const hotrg_result* r = &rr[(size_t)3 * j];
            cv[j] = beta * beta * (r[1].lnz_per_site - 2.0 * r[0].lnz_per_site + r[2].lnz_per_site) /
                    (opts->hb * opts->hb);
        }
    }
    std::vector<double> tp((size_t)n_h, std::nan(""));
    if (n_h > 0) {
        // (hbar + dh, hbar - dh) per (hbar, T), the other field zero
        std::vector<hotrg_params> pp((size_t)2 * n_h * n_t, q);
        std::vector<hotrg_result> rr;
        for (int k = 0; k < n_h; ++k)
            for (int j = 0; j < n_t; ++j) {
                hotrg_params* p = &pp[((size_t)k * n_t + j) * 2];
                p[0].beta = p[1].beta = 1.0 / temps[j];
                if (kind == HOTRG_T_IMP_M) {
                    p[0].h = hbar[k] + opts->dh;
                    p[1].h = hbar[k] - opts->dh;
                } else {
                    p[0].h1 = hbar[k] + opts->dh;
                    p[1].h1 = hbar[k] - opts->dh;
                }
            }
        hotrg_status s = run(pp, kind, rr);
        if (s != HOTRG_OK) return s;
        for (size_t i = 0; i < (size_t)n_h * n_t; ++i)
            chi[i] = (rr[2 * i].imp_ratio - rr[2 * i + 1].imp_ratio) / (2.0 * opts->dh);
        for (int k = 0; k < n_h; ++k) {
            double xp, yp;
            int32_t nf = 0;
            if (hotrg_find_peaks(temps, chi + (size_t)k * n_t, n_t, opts->min_prominence, 1, &xp, &yp, nullptr,
                                 &nf) != HOTRG_OK)
                return ::hotrg::set_err(ctx, HOTRG_EINVAL, "phase scan: a chi value is not finite");
            if (nf > 0) tp[k] = xp;
        }
    }
    if (t_peak)
        for (int k = 0; k < n_h; ++k) t_peak[k] = tp[k];
    if (fit) {
        std::vector<double> hx, ty;
        for (int k = 0; k < n_h; ++k)
            if (std::isfinite(tp[k])) {
                hx.push_back(hbar[k]);
                ty.push_back(tp[k]);
            }
        if ((int)hx.size() >= 3 && distinct_count(hx.data(), (int)hx.size()) >= 3) {
            hotrg_status s = hotrg_fit_tc(hx.data(), ty.data(), (int32_t)hx.size(), opts->c_lo, opts->c_hi, fit);
            if (s == HOTRG_ENOCONV)
                return ::hotrg::set_err(ctx, s, "phase scan: the zero-field fit found no stationary point");
            if (s != HOTRG_OK) return ::hotrg::set_err(ctx, s, "phase scan: zero-field fit rejected its input");
        }
    }
    return HOTRG_OK;
}

}  // extern "C"
