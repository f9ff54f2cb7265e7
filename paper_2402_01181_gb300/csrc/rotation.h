// rotation.h -- host-side tool-pose arithmetic (internal): unit quaternions,
// the rotation-vector maps, the frame a tool has inside one mpm_step call,
// and a forward-mode dual number so that the same code yields the frame's
// derivatives with respect to the two poses of the call.
#pragma once

#include <cmath>

namespace gbmpm {

inline double value_of(double x) { return x; }

// A value with its derivatives along N input directions.
template <int N>
struct Dual {
    double v = 0.0;
    double d[N] = {};
    Dual() = default;
    Dual(double x) : v(x) {}   // a constant
};
template <int N>
inline double value_of(const Dual<N> &x) { return x.v; }

template <int N>
inline Dual<N> operator+(const Dual<N> &a, const Dual<N> &b) {
    Dual<N> r(a.v + b.v);
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <int N>
inline Dual<N> operator-(const Dual<N> &a, const Dual<N> &b) {
    Dual<N> r(a.v - b.v);
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <int N>
inline Dual<N> operator-(const Dual<N> &a) {
    Dual<N> r(-a.v);
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
}
template <int N>
inline Dual<N> operator*(const Dual<N> &a, const Dual<N> &b) {
    Dual<N> r(a.v * b.v);
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
template <int N>
inline Dual<N> operator/(const Dual<N> &a, const Dual<N> &b) {
    Dual<N> r(a.v / b.v);
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
    return r;
}
template <int N> inline Dual<N> operator+(const Dual<N> &a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator+(double a, const Dual<N> &b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator-(const Dual<N> &a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N> &b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator*(const Dual<N> &a, double b) { return a * Dual<N>(b); }
template <int N> inline Dual<N> operator*(double a, const Dual<N> &b) { return Dual<N>(a) * b; }
template <int N> inline Dual<N> operator/(const Dual<N> &a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N> &b) { return Dual<N>(a) / b; }

template <int N>
inline Dual<N> chain(const Dual<N> &a, double f, double df) {   // f(a) with f'(a) = df
    Dual<N> r(f);
    for (int i = 0; i < N; ++i) r.d[i] = df * a.d[i];
    return r;
}
template <int N>
inline Dual<N> sqrt(const Dual<N> &a) {
    const double s = std::sqrt(a.v);
    return chain(a, s, 0.5 / s);
}
template <int N>
inline Dual<N> sin(const Dual<N> &a) { return chain(a, std::sin(a.v), std::cos(a.v)); }
template <int N>
inline Dual<N> cos(const Dual<N> &a) { return chain(a, std::cos(a.v), -std::sin(a.v)); }
template <int N>
inline Dual<N> atan2(const Dual<N> &y, const Dual<N> &x) {
    Dual<N> r(std::atan2(y.v, x.v));
    const double q = x.v * x.v + y.v * y.v;
    for (int i = 0; i < N; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / q;
    return r;
}

template <class S>
struct QuatT {
    S w, x, y, z;
};

template <class S>
QuatT<S> qmul(const QuatT<S> &a, const QuatT<S> &b) {
    return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z, a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
            a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x, a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}

// Unit quaternion of the rotation vector r.
template <class S>
QuatT<S> qexp_rotvec(const S r[3]) {
    using std::cos;
    using std::sin;
    using std::sqrt;
    const S th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    if (value_of(th2) < 1e-24) {
        const QuatT<S> q{S(1.0), 0.5 * r[0], 0.5 * r[1], 0.5 * r[2]};
        const S nq = sqrt(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
        return {q.w / nq, q.x / nq, q.y / nq, q.z / nq};
    }
    const S th = sqrt(th2);
    const S s = sin(0.5 * th) / th;
    return {cos(0.5 * th), s * r[0], s * r[1], s * r[2]};
}

// Rotation vector of the shortest rotation q represents.
template <class S>
void qlog_rotvec(QuatT<S> q, S r[3]) {
    using std::atan2;
    using std::sqrt;
    if (value_of(q.w) < 0) { q.w = -q.w; q.x = -q.x; q.y = -q.y; q.z = -q.z; }
    const S v2 = q.x * q.x + q.y * q.y + q.z * q.z;
    if (value_of(v2) < 1e-24) { r[0] = 2.0 * q.x; r[1] = 2.0 * q.y; r[2] = 2.0 * q.z; return; }
    const S v = sqrt(v2);
    const S th = 2.0 * atan2(v, q.w);
    r[0] = th * q.x / v; r[1] = th * q.y / v; r[2] = th * q.z / v;
}

template <class S>
void qmatrix(const QuatT<S> &q, S R[9]) {
    const S w = q.w, x = q.x, y = q.y, z = q.z;
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z); R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z); R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y); R[7] = 2.0 * (y * z + w * x); R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// The frame of a tool at fraction s in (0, 1] of a call that moves it
// uniformly from pose0 to pose1 (T, rotation vector) in span seconds:
// T(s) = T0 + s (T1 - T0), R(s) = exp(s phi) R0 with phi = log(R1 R0^T), and
// the rigid velocity u = (T1 - T0) / span, w = phi / span.
template <class S>
void call_frame(const S pose0[6], const S pose1[6], double s, double span, S R[9], S T[3], S u[3], S w[3]) {
    const QuatT<S> q0 = qexp_rotvec(pose0 + 3), q1 = qexp_rotvec(pose1 + 3);
    const QuatT<S> dq = qmul(q1, QuatT<S>{q0.w, -q0.x, -q0.y, -q0.z});
    S phi[3];
    qlog_rotvec(dq, phi);
    const S rs[3] = {s * phi[0], s * phi[1], s * phi[2]};
    qmatrix(qmul(qexp_rotvec(rs), q0), R);
    for (int a = 0; a < 3; ++a) {
        T[a] = pose0[a] + s * (pose1[a] - pose0[a]);
        u[a] = (pose1[a] - pose0[a]) / span;
        w[a] = phi[a] / span;
    }
}

}  // namespace gbmpm
