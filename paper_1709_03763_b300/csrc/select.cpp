// Host pose utilities.  Keyframe selection for re-integration (Section 4.3): the pose distance
// ||s t - s t'|| with s = (2,2,2,1,1,1), BundleFusion's m most-moved keyframes,
// and Eq. 3's m most-moved *consecutive* keyframes.  Host code: K is the number
// of keyframes (hundreds to thousands), far too small for a GPU launch.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "surfcorr.h"

namespace {

// Z-Y-X Euler angles (yaw about z, pitch about y, roll about x) of R = Rz Ry Rx.
void euler_zyx(const sc_pose& T, double e[3]) {
    const double r20 = std::max(-1.0, std::min(1.0, (double)T.m[2][0]));
    e[0] = std::atan2((double)T.m[1][0], (double)T.m[0][0]);
    e[1] = std::asin(-r20);
    e[2] = std::atan2((double)T.m[2][1], (double)T.m[2][2]);
}

double wrap_pi(double a) {
    const double two_pi = 6.283185307179586476925;
    a = std::fmod(a, two_pi);
    if (a > 3.14159265358979323846) a -= two_pi;
    if (a <= -3.14159265358979323846) a += two_pi;
    return a;
}

}  // namespace

extern "C" double sc_pose_distance(const sc_pose* a, const sc_pose* b) {
    if (!a || !b) return NAN;
    double ea[3], eb[3];
    euler_zyx(*a, ea);
    euler_zyx(*b, eb);
    double s2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double d = 2.0 * wrap_pi(ea[k] - eb[k]);
        s2 += d * d;
    }
    for (int k = 0; k < 3; ++k) {
        const double d = (double)a->m[k][3] - (double)b->m[k][3];
        s2 += d * d;
    }
    return std::sqrt(s2);
}

extern "C" int sc_select_topm(const double* dist, int32_t K, int32_t m, int32_t* out) {
    if (!dist || !out || K < 0 || m < 0) return SC_ERR_INVALID_ARG;
    std::vector<int32_t> order(K);
    std::iota(order.begin(), order.end(), 0);
    // descending distance; equal distances keep ascending index order
    std::stable_sort(order.begin(), order.end(), [&](int32_t i, int32_t j) { return dist[i] > dist[j]; });
    const int32_t take = std::min(m, K);
    for (int32_t i = 0; i < take; ++i) out[i] = order[i];
    return SC_OK;
}

extern "C" int sc_select_consecutive(const double* dist, int32_t K, int32_t m) {
    if (!dist || m < 1 || K < m) return SC_ERR_INVALID_ARG;
    // each window summed from scratch (no running-sum drift); strict '>' keeps the
    // smallest j on ties
    double best = -1.0;
    int32_t jbest = 0;
    for (int32_t j = 0; j + m <= K; ++j) {
        double window = 0.0;
        for (int32_t i = j; i < j + m; ++i) window += dist[i];
        if (j == 0 || window > best) {
            best = window;
            jbest = j;
        }
    }
    return jbest;
}

// exp(xi^) T with xi = (rho, omega): R' = Exp(omega) R, t' = Exp(omega) t + V(omega) rho.
extern "C" int sc_pose_exp_left(const sc_pose* T, const double* xi, sc_pose* out) {
    if (!T || !xi || !out) return SC_ERR_INVALID_ARG;
    const double* w = xi + 3;
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double th = std::sqrt(th2);
    double a, b, c;  // sin(th)/th, (1-cos th)/th^2, (th - sin th)/th^3
    if (th < 1e-6) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
        c = 1.0 / 6.0 - th2 / 120.0;
    } else {
        a = std::sin(th) / th;
        b = (1.0 - std::cos(th)) / th2;
        c = (th - std::sin(th)) / (th2 * th);
    }
    const double K[3][3] = {{0, -w[2], w[1]}, {w[2], 0, -w[0]}, {-w[1], w[0], 0}};
    double K2[3][3], R[3][3], Vm[3][3];
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            K2[r][q] = 0;
            for (int k = 0; k < 3; ++k) K2[r][q] += K[r][k] * K[k][q];
        }
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            const double I = r == q ? 1.0 : 0.0;
            R[r][q] = I + a * K[r][q] + b * K2[r][q];
            Vm[r][q] = I + b * K[r][q] + c * K2[r][q];
        }
    sc_pose o;
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[r][k] * (double)T->m[k][q];
            o.m[r][q] = (float)acc;
        }
        double acc = 0;
        for (int k = 0; k < 3; ++k) acc += R[r][k] * (double)T->m[k][3] + Vm[r][k] * xi[k];
        o.m[r][3] = (float)acc;
    }
    *out = o;
    return SC_OK;
}
