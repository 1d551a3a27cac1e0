// Surrogate driver: standardisation, training, prediction, refinement points
// near the C_V / chi maxima, and re-solving uncertain points with HOTRG.
// Host C++ over the MLP kernels (hotrg_mlp.cu) and the batched observables
// (hotrg_api.cu); the thesis has no counterpart.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace {

void standardise_x(const hotrg_scaling* s, const double* X, int32_t n, std::vector<float>& out) {
    out.resize((size_t)n * 2);
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 2; ++c) out[i * 2 + c] = (float)((X[i * 2 + c] - s->x_mean[c]) / s->x_std[c]);
}

bool finite_scaling(const hotrg_scaling* s) {
    for (int c = 0; c < 2; ++c)
        if (!std::isfinite(s->x_mean[c]) || !(s->x_std[c] > 0) || !std::isfinite(s->x_std[c])) return false;
    for (int c = 0; c < 4; ++c)
        if (!std::isfinite(s->y_mean[c]) || !(s->y_std[c] > 0) || !std::isfinite(s->y_std[c])) return false;
    return true;
}

}  // namespace

extern "C" {

hotrg_status hotrg_scaling_fit(const double* X, const double* Y, int32_t n, hotrg_scaling* s) {
    if (!X || !Y || !s || n < 1) return HOTRG_EINVAL;
    auto col = [n](const double* A, int w, int c, double& mean, double& sd) {
        double m = 0.0;
        for (int64_t i = 0; i < n; ++i) m += A[i * w + c];
        m /= n;
        double v = 0.0;
        for (int64_t i = 0; i < n; ++i) v += (A[i * w + c] - m) * (A[i * w + c] - m);
        v /= n;
        mean = m;
        sd = v > 0.0 ? std::sqrt(v) : 1.0;
    };
    for (int c = 0; c < 2; ++c) col(X, 2, c, s->x_mean[c], s->x_std[c]);
    for (int c = 0; c < 4; ++c) col(Y, 4, c, s->y_mean[c], s->y_std[c]);
    return finite_scaling(s) ? HOTRG_OK : HOTRG_EINVAL;
}

hotrg_status hotrg_surrogate_fit(hotrg_mlp* m, const double* X, const double* Y, int32_t n, int32_t epochs,
                                 int32_t batch, float lr, hotrg_scaling* s, float* final_loss) {
    if (!m || !X || !Y || !s || n < 1) return HOTRG_EINVAL;
    hotrg_status st = hotrg_scaling_fit(X, Y, n, s);
    if (st != HOTRG_OK) return st;
    std::vector<float> xs, ys((size_t)n * 4);
    standardise_x(s, X, n, xs);
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 4; ++c) ys[i * 4 + c] = (float)((Y[i * 4 + c] - s->y_mean[c]) / s->y_std[c]);
    return hotrg_mlp_train(m, xs.data(), ys.data(), n, epochs, batch, lr, final_loss);
}

hotrg_status hotrg_surrogate_predict(hotrg_mlp* m, const hotrg_scaling* s, const double* X, int32_t n, double* y,
                                     double* spread) {
    if (!m || !s || !X || !y || n < 0 || !finite_scaling(s)) return HOTRG_EINVAL;
    if (n == 0) return HOTRG_OK;
    std::vector<float> xs, mean((size_t)n * 4), sd((size_t)n * 4);
    standardise_x(s, X, n, xs);
    hotrg_status st = hotrg_mlp_predict(m, xs.data(), n, mean.data(), sd.data());
    if (st != HOTRG_OK) return st;
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 4; ++c) {
            y[i * 4 + c] = (double)mean[i * 4 + c] * s->y_std[c] + s->y_mean[c];
            if (spread) spread[i * 4 + c] = (double)sd[i * 4 + c];
        }
    return HOTRG_OK;
}

hotrg_status hotrg_surrogate_peaks(hotrg_mlp* m, const hotrg_scaling* s, const double* deltas, int32_t n_delta,
                                   double beta_lo, double beta_hi, int32_t n_beta, int32_t per_peak, double width,
                                   double* X_out, double* peaks_out) {
    if (!m || !s || !deltas || !X_out || n_delta < 1 || n_beta < 2 || per_peak < 1 || !(beta_hi > beta_lo) ||
        !(width >= 0))
        return HOTRG_EINVAL;
    const int64_t n = (int64_t)n_delta * n_beta;
    if (n > (int64_t)1 << 26) return HOTRG_EINVAL;
    std::vector<double> X((size_t)n * 2), Y((size_t)n * 4);
    const double db = (beta_hi - beta_lo) / (n_beta - 1);
    for (int64_t a = 0; a < n_delta; ++a)
        for (int64_t b = 0; b < n_beta; ++b) {
            X[(a * n_beta + b) * 2 + 0] = beta_lo + db * b;
            X[(a * n_beta + b) * 2 + 1] = deltas[a];
        }
    hotrg_status st = hotrg_surrogate_predict(m, s, X.data(), (int32_t)n, Y.data(), nullptr);
    if (st != HOTRG_OK) return st;
    int64_t row = 0;
    for (int64_t a = 0; a < n_delta; ++a)
        for (int o = 1; o <= 2; ++o) {  // 1: C_V, 2: chi
            int64_t best = 0;
            for (int64_t b = 1; b < n_beta; ++b)
                if (Y[(a * n_beta + b) * 4 + o] > Y[(a * n_beta + best) * 4 + o]) best = b;
            const double bstar = beta_lo + db * best;
            if (peaks_out) peaks_out[a * 2 + (o - 1)] = bstar;
            const double lo = std::max(beta_lo, bstar - width), hi = std::min(beta_hi, bstar + width);
            for (int j = 0; j < per_peak; ++j, ++row) {
                X_out[row * 2 + 0] = per_peak == 1 ? bstar : lo + (hi - lo) * j / (per_peak - 1);
                X_out[row * 2 + 1] = deltas[a];
            }
        }
    return HOTRG_OK;
}

hotrg_status hotrg_surrogate_refine(hotrg_ctx* ctx, hotrg_mlp* m, const hotrg_scaling* s, const hotrg_params* base,
                                    const double* X, int32_t n, double threshold, double hb, double hbar, double dh,
                                    int32_t nstreams, double* y, double* spread, int32_t* solved,
                                    int32_t* n_solved) {
    if (!ctx || !m || !s || !base || !X || !y || !solved || n < 0 || !(threshold >= 0)) return HOTRG_EINVAL;
    std::vector<double> sd((size_t)n * 4);
    hotrg_status st = hotrg_surrogate_predict(m, s, X, n, y, sd.data());
    if (st != HOTRG_OK) return st;
    std::vector<int> idx;
    for (int64_t i = 0; i < n; ++i) {
        double w = 0.0;
        for (int c = 0; c < 4; ++c) w = std::max(w, sd[i * 4 + c]);
        solved[i] = w > threshold ? 1 : 0;
        if (solved[i]) idx.push_back((int)i);
        if (spread)
            for (int c = 0; c < 4; ++c) spread[i * 4 + c] = sd[i * 4 + c];
    }
    if (n_solved) *n_solved = (int32_t)idx.size();
    if (idx.empty()) return HOTRG_OK;
    std::vector<hotrg_params> pp(idx.size(), *base);
    for (size_t k = 0; k < idx.size(); ++k) {
        pp[k].beta = X[(size_t)idx[k] * 2 + 0];
        pp[k].delta = X[(size_t)idx[k] * 2 + 1];
    }
    std::vector<hotrg_obs> ob(idx.size());
    st = hotrg_observables_batch(ctx, pp.data(), (int32_t)idx.size(), hb, hbar, dh, nstreams, ob.data());
    if (st != HOTRG_OK) return st;
    for (size_t k = 0; k < idx.size(); ++k) {
        double* r = y + (size_t)idx[k] * 4;
        r[0] = ob[k].f;
        r[1] = ob[k].cv;
        r[2] = ob[k].chi;
        r[3] = ob[k].chi1;
    }
    return HOTRG_OK;
}

}  // extern "C"
