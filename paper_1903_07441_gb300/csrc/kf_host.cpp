// Constant-velocity Kalman filter for obstacle tracks (Sec. 3.5, Eqs. 7-13).
// Host code: 200-300 tracks x a 4x4 update per frame is microseconds of CPU
// work and off the hot path; the predicted poses it feeds are evaluated on the
// GPU by tw_build_grid.
//
// The structure of the model is used directly: A = [[I, dt I], [0, I]] and
// H = [I 0], so A P A^T, the 2x2 innovation covariance and the gain are
// written out in blocks rather than as general matrix products.
#include <math.h>
#include <string.h>

#include "twgrid.h"

namespace {

bool all_finite(const double *v, int n) {
    for (int i = 0; i < n; i++)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// P <- A P A^T + Q(dt) for A = [[I, dt I], [0, I]] (4x4 row-major, state x, y, vx, vy).
void predict_cov(double P[16], double dt, double q) {
    double M[16];
    // M = A P: rows 0,1 gain dt * rows 2,3
    for (int j = 0; j < 4; j++) {
        M[0 * 4 + j] = P[0 * 4 + j] + dt * P[2 * 4 + j];
        M[1 * 4 + j] = P[1 * 4 + j] + dt * P[3 * 4 + j];
        M[2 * 4 + j] = P[2 * 4 + j];
        M[3 * 4 + j] = P[3 * 4 + j];
    }
    // P = M A^T: columns 0,1 gain dt * columns 2,3
    for (int i = 0; i < 4; i++) {
        P[i * 4 + 0] = M[i * 4 + 0] + dt * M[i * 4 + 2];
        P[i * 4 + 1] = M[i * 4 + 1] + dt * M[i * 4 + 3];
        P[i * 4 + 2] = M[i * 4 + 2];
        P[i * 4 + 3] = M[i * 4 + 3];
    }
    const double a = q * dt * dt * dt / 3.0, b = q * dt * dt / 2.0, c = q * dt;
    P[0] += a; P[5] += a; P[10] += c; P[15] += c;
    P[2] += b; P[8] += b; P[7] += b; P[13] += b;
}

}  // namespace

extern "C" int kf_init(tw_track *tracks, int n, const double *z, const double *radius, double r_meas,
                       double p_vel) {
    if (n < 0 || (n > 0 && (!tracks || !z || !radius)) || !std::isfinite(r_meas) || r_meas <= 0.0 ||
        !std::isfinite(p_vel) || p_vel < 0.0)
        return TW_EINVAL;
    for (int o = 0; o < n; o++) {
        tw_track &T = tracks[o];
        if (!all_finite(z + 2 * o, 2) || !std::isfinite(radius[o]) || radius[o] < 0.0) return TW_EINVAL;
        memset(&T, 0, sizeof(T));
        T.x[0] = z[2 * o];
        T.x[1] = z[2 * o + 1];
        T.P[0] = T.P[5] = r_meas * r_meas;
        T.P[10] = T.P[15] = p_vel;
        T.radius = radius[o];
    }
    return TW_OK;
}

extern "C" int kf_update(tw_track *tracks, int n, const double *z, double dt, double q_accel, double r_meas) {
    if (n < 0 || (n > 0 && (!tracks || !z)) || !std::isfinite(dt) || dt < 0.0 || !std::isfinite(q_accel) ||
        q_accel < 0.0 || !std::isfinite(r_meas) || r_meas <= 0.0)
        return TW_EINVAL;
    for (int o = 0; o < n; o++)
        if (!all_finite(tracks[o].x, 4) || !all_finite(tracks[o].P, 16) || !all_finite(z + 2 * o, 2))
            return TW_EINVAL;
    const double r2 = r_meas * r_meas;
    for (int o = 0; o < n; o++) {
        double *x = tracks[o].x, *P = tracks[o].P;
        // predict (Eqs. 9-10)
        x[0] += dt * x[2];
        x[1] += dt * x[3];
        predict_cov(P, dt, q_accel);
        // innovation covariance S = H P H^T + R (top-left 2x2 block of P plus R)
        double s00 = P[0] + r2, s01 = P[1], s10 = P[4], s11 = P[5] + r2;
        double det = s00 * s11 - s01 * s10;
        if (!(det > 0.0)) return TW_EINVAL;
        double i00 = s11 / det, i01 = -s01 / det, i10 = -s10 / det, i11 = s00 / det;
        // gain K = P H^T S^-1 (Eq. 13): columns 0,1 of P times S^-1
        double K[4][2];
        for (int i = 0; i < 4; i++) {
            K[i][0] = P[i * 4 + 0] * i00 + P[i * 4 + 1] * i10;
            K[i][1] = P[i * 4 + 0] * i01 + P[i * 4 + 1] * i11;
        }
        // state (Eq. 11)
        const double y0 = z[2 * o] - x[0], y1 = z[2 * o + 1] - x[1];
        for (int i = 0; i < 4; i++) x[i] += K[i][0] * y0 + K[i][1] * y1;
        // covariance (Eq. 12): P <- P - K (H P), H P = rows 0,1 of P
        double HP[2][4];
        for (int j = 0; j < 4; j++) { HP[0][j] = P[j]; HP[1][j] = P[4 + j]; }
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) P[i * 4 + j] -= K[i][0] * HP[0][j] + K[i][1] * HP[1][j];
    }
    return TW_OK;
}
