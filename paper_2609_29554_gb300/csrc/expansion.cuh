// Device arithmetic on non-overlapping expansions of N binary64 components
// (DD N = 2, TD N = 3, QD N = 4; Sec. 2.1), built from the error-free
// transformations TwoSum and TwoProd (FMA).  Used by the panel's column
// kernels where the cooperative base-block kernel does not apply (its rows do
// not fit in shared memory) and by the native per-element LU baseline.
//
// Products and sums are formed order by order: terms of order k (about
// 2^(-53 k) relative to the leading one) are added with TwoSum, each rounding
// error moving to order k + 1; order N - 1 is summed plainly, then the N
// leading values are renormalised.  The error is a few units of 2^(-53 N)
// relative to the operands' magnitude.
#pragma once

namespace ozlu {

template <int N>
struct Exp {
    double x[N];
};

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
    p = a * b;
    e = fma(a, b, -p);
}

// Renormalise v[0..M) (ordered by decreasing order of magnitude, overlapping
// allowed) into N non-overlapping components.
template <int N, int M>
__device__ __forceinline__ Exp<N> renorm(double (&v)[M]) {
    // bottom-up TwoSum sweep: s carries the running sum, v[i] keeps the errors
    double s = v[M - 1];
#pragma unroll
    for (int i = M - 2; i >= 0; --i) {
        double e;
        two_sum(v[i], s, s, e);
        v[i + 1] = e;
    }
    v[0] = s;
    // top-down: emit a component whenever the carried error is nonzero
    Exp<N> r;
#pragma unroll
    for (int i = 0; i < N; ++i) r.x[i] = 0.0;
    double cur = v[0];
    int k = 0;
#pragma unroll
    for (int i = 1; i < M; ++i) {
        double s2, e2;
        fast_two_sum(cur, v[i], s2, e2);
        if (e2 != 0.0) {
            if (k < N) r.x[k] = s2;
            ++k;
            cur = e2;
        } else {
            cur = s2;
        }
    }
    if (k < N) r.x[k] = cur;
    return r;
}

template <int N>
__device__ __forceinline__ Exp<N> neg(const Exp<N>& a) {
    Exp<N> r;
#pragma unroll
    for (int i = 0; i < N; ++i) r.x[i] = -a.x[i];
    return r;
}

template <int N>
__device__ __forceinline__ Exp<N> add(const Exp<N>& a, const Exp<N>& b) {
    // order k holds a_k, b_k and the TwoSum errors of order k - 1
    double out[N + 1];
    double carry[2 * N];
    int nc = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double s = a.x[k];
        double nxt[2 * N];
        int nn = 0;
        double e;
        two_sum(s, b.x[k], s, e);
        nxt[nn++] = e;
#pragma unroll
        for (int j = 0; j < 2 * N; ++j) {
            if (j < nc) {
                if (k < N - 1) {
                    two_sum(s, carry[j], s, e);
                    nxt[nn++] = e;
                } else {
                    s += carry[j];
                }
            }
        }
        out[k] = s;
        nc = 0;
#pragma unroll
        for (int j = 0; j < 2 * N; ++j)
            if (j < nn && k < N - 1) carry[nc++] = nxt[j];
        if (k == N - 1) {
            double rest = 0.0;
#pragma unroll
            for (int j = 0; j < 2 * N; ++j)
                if (j < nn) rest += nxt[j];
            out[N] = rest;
        }
    }
    return renorm<N, N + 1>(out);
}

template <int N>
__device__ __forceinline__ Exp<N> sub(const Exp<N>& a, const Exp<N>& b) {
    return add<N>(a, neg<N>(b));
}

template <int N>
__device__ __forceinline__ Exp<N> mul(const Exp<N>& a, const Exp<N>& b) {
    // terms[k]: order-k contributions; TwoProd errors and TwoSum errors move up
    constexpr int CAP = 4 * N * N;
    double cur[CAP];
    int ncur = 0;
    double out[N + 1];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double nxt[CAP];
        int nn = 0;
        double s = 0.0;
        bool first = true;
#pragma unroll
        for (int i = 0; i <= k; ++i) {
            const int j = k - i;
            if (k < N - 1) {
                double p, e;
                two_prod(a.x[i], b.x[j], p, e);
                nxt[nn++] = e;
                if (first) { s = p; first = false; }
                else { double e2; two_sum(s, p, s, e2); nxt[nn++] = e2; }
            } else {
                s += a.x[i] * b.x[j];
            }
        }
#pragma unroll
        for (int t = 0; t < CAP; ++t) {
            if (t < ncur) {
                if (k < N - 1) { double e2; two_sum(s, cur[t], s, e2); nxt[nn++] = e2; }
                else s += cur[t];
            }
        }
        out[k] = s;
        ncur = 0;
        if (k < N - 1) {
#pragma unroll
            for (int t = 0; t < CAP; ++t)
                if (t < nn) cur[ncur++] = nxt[t];
        }
    }
    // order N: products a_i b_j with i + j = N (no error terms needed)
    double tail = 0.0;
#pragma unroll
    for (int i = 1; i < N; ++i) tail += a.x[i] * b.x[N - i];
    out[N] = tail;
    return renorm<N, N + 1>(out);
}

// a * d for a double d
template <int N>
__device__ __forceinline__ Exp<N> mul_d(const Exp<N>& a, double d) {
    Exp<N> b;
    b.x[0] = d;
#pragma unroll
    for (int i = 1; i < N; ++i) b.x[i] = 0.0;
    return mul<N>(a, b);
}

// a / b by long division: N + 1 quotient digits, renormalised
template <int N>
__device__ __forceinline__ Exp<N> div(const Exp<N>& a, const Exp<N>& b) {
    double q[N + 1];
    Exp<N> r = a;
#pragma unroll
    for (int i = 0; i <= N; ++i) {
        q[i] = r.x[0] / b.x[0];
        if (i < N) r = sub<N>(r, mul_d<N>(b, q[i]));
    }
    return renorm<N, N + 1>(q);
}

// c - a * b
template <int N>
__device__ __forceinline__ Exp<N> fms(const Exp<N>& c, const Exp<N>& a, const Exp<N>& b) {
    return sub<N>(c, mul<N>(a, b));
}

// compare |a| with |b|: -1, 0, +1 (component by component after sign normalisation)
template <int N>
__device__ __forceinline__ int abs_cmp(const Exp<N>& a, const Exp<N>& b) {
    const double sa = a.x[0] < 0 ? -1.0 : 1.0, sb = b.x[0] < 0 ? -1.0 : 1.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const double u = sa * a.x[i], v = sb * b.x[i];
        if (u > v) return 1;
        if (u < v) return -1;
    }
    return 0;
}

template <int N>
__device__ __forceinline__ Exp<N> load(const double* p) {
    Exp<N> r;
#pragma unroll
    for (int i = 0; i < N; ++i) r.x[i] = p[i];
    return r;
}

template <int N>
__device__ __forceinline__ void store(double* p, const Exp<N>& v) {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = v.x[i];
}

template <int N>
__device__ __forceinline__ bool is_zero(const Exp<N>& a) {
    return a.x[0] == 0.0;
}

}  // namespace ozlu
