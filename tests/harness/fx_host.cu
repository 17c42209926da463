// Test harness: the integer-digit arithmetic of csrc/fx.cuh compiled for the
// host, with a C interface, so that the tests can compare it with exact
// rational arithmetic.  Arrays of multiple doubles are limb-planar:
// x[l * n + i] is limb l of entry i.
#include <vector>

#include "../../paper_2110_08375_gb300/csrc/fx.cuh"

using namespace mdls;
using namespace mdls::fx;

template <int P>
static md<P> load(const double* x, long n, long i) {
    md<P> r;
    for (int l = 0; l < P; ++l) r.v[l] = x[l * n + i];
    return r;
}

template <int P>
static void store(double* x, long n, long i, const md<P>& r) {
    for (int l = 0; l < P; ++l) x[l * n + i] = r.v[l];
}

// op: 0 roundtrip, 1 mul, 2 add, 3 sub, 4 recip, 5 rsqrt, 6 sqrt (a * rsqrt a),
// 7 a * 2^-1 (bit shift), 8 a * 2^5
template <int P>
static void scalar_ops(int op, long n, const double* a, const double* b, double* c) {
    constexpr int N = Cfg<P>::N;
    for (long i = 0; i < n; ++i) {
        const xf<N> x = xf_from_md<P, N>(load<P>(a, n, i));
        const xf<N> y = xf_from_md<P, N>(load<P>(b, n, i));
        xf<N> r;
        switch (op) {
            case 0: r = x; break;
            case 1: r = xf_mul<N>(x, y); break;
            case 2: r = xf_add<N>(x, y); break;
            case 3: r = xf_sub<N>(x, y); break;
            case 4: r = xf_recip<N>(x); break;
            case 5: r = xf_rsqrt<N>(x); break;
            case 6: r = xf_mul<N>(x, xf_rsqrt<N>(x)); break;
            case 7: r = xf_shift_bits<N>(x, -1); break;
            default: r = xf_shift_bits<N>(x, 5); break;
        }
        store<P>(c, n, i, xf_to_md<P, N>(r));
    }
}

extern "C" int fx_digits(int p, int which) {
    if (p == 2) return which ? Cfg<2>::N : Cfg<2>::D;
    if (p == 4) return which ? Cfg<4>::N : Cfg<4>::D;
    return which ? Cfg<8>::N : Cfg<8>::D;
}

extern "C" void fx_scalar(int p, int op, long n, const double* a, const double* b, double* c) {
    if (p == 2) scalar_ops<2>(op, n, a, b, c);
    else if (p == 4) scalar_ops<4>(op, n, a, b, c);
    else scalar_ops<8>(op, n, a, b, c);
}

// Fixed point at digit scale e: x -> digits -> md (through a scalar).
template <int P>
static void fixed_roundtrip(long n, const double* x, int e, double* y, int32_t* digits) {
    constexpr int D = Cfg<P>::D, N = Cfg<P>::N;
    for (long i = 0; i < n; ++i) {
        int32_t d[D];
        fixed_from_md<P, D>(load<P>(x, n, i), e, d);
        for (int k = 0; k < D; ++k) digits[k * n + i] = d[k];
        store<P>(y, n, i, xf_to_md<P, N>(xf_from_fixed<N, D>(d, e)));
    }
}

extern "C" void fx_fixed_roundtrip(int p, long n, const double* x, int e, double* y, int32_t* digits) {
    if (p == 2) fixed_roundtrip<2>(n, x, e, y, digits);
    else if (p == 4) fixed_roundtrip<4>(n, x, e, y, digits);
    else fixed_roundtrip<8>(n, x, e, y, digits);
}

// sum_i u_i a_i (mode 0) or sum_i a_i^2 (mode 1) with u at scale eu, a at
// scale ea, accumulated by diagonals; the result as one md.
template <int P>
static void dot(int mode, long n, const double* u, const double* a, int eu, int ea, double* out) {
    constexpr int D = Cfg<P>::D, N = Cfg<P>::N;
    int64_t acc[D + 3];
    for (int k = 0; k < D + 3; ++k) acc[k] = 0;
    for (long i = 0; i < n; ++i) {
        int32_t du[D], da[D];
        fixed_from_md<P, D>(load<P>(a, n, i), ea, da);
        if (mode == 0) {
            fixed_from_md<P, D>(load<P>(u, n, i), eu, du);
            dot_acc<D>(du, da, acc);
        } else {
            dot_acc<D>(da, da, acc);
        }
    }
    const int e0 = (mode == 0 ? eu : ea) + ea + D - 3;
    store<P>(out, 1, 0, xf_to_md<P, N>(xf_from_acc<N>(acc, e0)));
}

extern "C" void fx_dot(int p, int mode, long n, const double* u, const double* a, int eu, int ea, double* out) {
    if (p == 2) dot<2>(mode, n, u, a, eu, ea, out);
    else if (p == 4) dot<4>(mode, n, u, a, eu, ea, out);
    else dot<8>(mode, n, u, a, eu, ea, out);
}

// a_i -= w u_i for every i: a at scale ea, u at scale eu, w a scalar turned
// into two integer and D-2 fractional digits of w 2^(24(eu-ea)).  Returns 0
// if w does not fit.
template <int P>
static int axpy(long n, double* a, const double* u, const double* w, int ea, int eu) {
    constexpr int D = Cfg<P>::D, N = Cfg<P>::N;
    const xf<N> W = xf_from_md<P, N>(load<P>(w, 1, 0));
    int32_t dw[D];
    if (!fixed_from_xf<N, D>(W, ea - eu - (D - 2), dw)) return 0;
    for (long i = 0; i < n; ++i) {
        int32_t du[D], da[D];
        fixed_from_md<P, D>(load<P>(a, n, i), ea, da);
        fixed_from_md<P, D>(load<P>(u, n, i), eu, du);
        axpy_row<D>(da, dw, du);
        store<P>(a, n, i, xf_to_md<P, N>(xf_from_fixed<N, D>(da, ea)));
    }
    return 1;
}

extern "C" int fx_axpy(int p, long n, double* a, const double* u, const double* w, int ea, int eu) {
    if (p == 2) return axpy<2>(n, a, u, w, ea, eu);
    if (p == 4) return axpy<4>(n, a, u, w, ea, eu);
    return axpy<8>(n, a, u, w, ea, eu);
}

// Householder scalars from sigma and x0 (entries i): v0, bp, R, 1/v0, beta
// and the kind.
// variant 0: digits (xf_house); 1: the P-limb FP64 form (xf_house_md);
// 2: the short-chain double double form the panels run (xf_house_dd, P = 2).
template <int P>
static void house(long n, const double* sig, const double* x0, double* v0, double* bp, double* rcc,
                  double* inv, double* beta, int* kind, int variant) {
    constexpr int N = Cfg<P>::N;
    for (long i = 0; i < n; ++i) {
        xf<N> V, B, R, I, Be;
        const xf<N> S = xf_from_md<P, N>(load<P>(sig, n, i)), X = xf_from_md<P, N>(load<P>(x0, n, i));
        kind[i] = variant == 2   ? xf_house_dd<N>(S, X, V, B, R, I, Be)
                  : variant == 1 ? xf_house_md<P, N>(S, X, V, B, R, I, Be)
                                 : xf_house<N>(S, X, V, B, R, I, Be);
        store<P>(v0, n, i, xf_to_md<P, N>(V));
        store<P>(bp, n, i, xf_to_md<P, N>(B));
        store<P>(rcc, n, i, xf_to_md<P, N>(R));
        store<P>(inv, n, i, xf_to_md<P, N>(I));
        store<P>(beta, n, i, xf_to_md<P, N>(Be));
    }
}

extern "C" void fx_house(int p, long n, const double* sig, const double* x0, double* v0, double* bp,
                         double* rcc, double* inv, double* beta, int* kind) {
    if (p == 2) house<2>(n, sig, x0, v0, bp, rcc, inv, beta, kind, 0);
    else if (p == 4) house<4>(n, sig, x0, v0, bp, rcc, inv, beta, kind, 0);
    else house<8>(n, sig, x0, v0, bp, rcc, inv, beta, kind, 0);
}

extern "C" void fx_house_md(int p, long n, const double* sig, const double* x0, double* v0, double* bp,
                            double* rcc, double* inv, double* beta, int* kind) {
    if (p == 2) house<2>(n, sig, x0, v0, bp, rcc, inv, beta, kind, 1);
    else if (p == 4) house<4>(n, sig, x0, v0, bp, rcc, inv, beta, kind, 1);
    else house<8>(n, sig, x0, v0, bp, rcc, inv, beta, kind, 1);
}

// double double only
extern "C" void fx_house_dd(long n, const double* sig, const double* x0, double* v0, double* bp, double* rcc,
                            double* inv, double* beta, int* kind) {
    house<2>(n, sig, x0, v0, bp, rcc, inv, beta, kind, 2);
}

// Sequential replay of the integer-digit panel (one panel of all n columns
// of an m x n matrix, column-major limb-planar, ld = m): the same scale,
// conversions, dot products, updates, rescaling and scalars as the device
// kernel, one column after the other.  A is overwritten with R (upper) and
// v (below the diagonal); beta receives the n betas.
template <int P>
static int panel_replay(long m, long n, double* A, double* beta) {
    constexpr int D = Cfg<P>::D, N = Cfg<P>::N, M = D + 3;
    const long ps = m * n;
    std::vector<int32_t> F((size_t)D * n * m);
    std::vector<int> ecs(n), eus(n), kinds(n);
    std::vector<xf<N>> v0s(n), bps(n);
    auto dig = [&](long c, long i, int k) -> int32_t& { return F[((size_t)k * n + c) * m + i]; };
    for (long c = 0; c < n; ++c) {
        double* col = A + c * m;
        // scale
        double mx = 0, ss = 0;
        for (long i = 0; i < m; ++i) mx = fmax(mx, fabs(col[i]));
        int ec = -D;
        if (mx > 0) {
            int emax;
            frexp(mx, &emax);
            emax -= 1;
            for (long i = 0; i < m; ++i) ss += ldexp(col[i], -emax) * ldexp(col[i], -emax);
            int k;
            frexp(sqrt(ss), &k);
            const int bound = emax + k + 1;
            ec = floordiv24(bound + 3 + kB - 1) - D;
        }
        ecs[c] = ec;
        for (long i = 0; i < m; ++i) {
            md<P> x;
            for (int l = 0; l < P; ++l) x.v[l] = col[l * ps + i];
            int32_t d[D];
            fixed_from_md<P, D>(x, ec, d);
            for (int k = 0; k < D; ++k) dig(c, i, k) = d[k];
        }
        for (long ell = 0; ell < c; ++ell) {
            const int eu = eus[ell];
            int64_t acc[M] = {};
            for (long i = ell + 1; i < m; ++i) {
                int32_t u[D], x[D];
                for (int k = 0; k < D; ++k) {
                    u[k] = dig(ell, i, k);
                    x[k] = dig(c, i, k);
                }
                dot_acc<D>(u, x, acc);
            }
            int32_t xe[D];
            for (int k = 0; k < D; ++k) xe[k] = dig(c, ell, k);
            const xf<N> x_ell = xf_from_fixed<N, D>(xe, ec);
            const xf<N> s = xf_add<N>(xf_from_acc<N>(acc, eu + ec + D - 3), xf_mul<N>(v0s[ell], x_ell));
            const xf<N> W = xf_mul<N>(bps[ell], s);
            if (!fixed_from_xf<N, D>(xf_sub<N>(x_ell, xf_mul<N>(W, v0s[ell])), ec, xe)) return 1;
            for (int k = 0; k < D; ++k) dig(c, ell, k) = xe[k];
            if (kinds[ell] != 0) continue;
            int32_t wd[D];
            if (!fixed_from_xf<N, D>(W, ec - eu - (D - 2), wd)) return 2;
            for (long i = ell + 1; i < m; ++i) {
                int32_t u[D], x[D];
                for (int k = 0; k < D; ++k) {
                    u[k] = dig(ell, i, k);
                    x[k] = dig(c, i, k);
                }
                axpy_row<D>(x, wd, u);
                for (int k = 0; k < D; ++k) dig(c, i, k) = x[k];
            }
        }
        int64_t sacc[M] = {};
        int top = -1;
        for (long i = c + 1; i < m; ++i) {
            int32_t x[D];
            for (int k = 0; k < D; ++k) x[k] = dig(c, i, k);
            dot_acc<D>(x, x, sacc);
            const int tp = fixed_top<D>(x);
            top = tp > top ? tp : top;
        }
        const int qsh = (top >= 0 && top < D - 2) ? D - 2 - top : 0;
        for (long i = c + 1; i < m; ++i)
            for (int k = D - 1; k >= 0; --k) dig(c, i, k) = k >= qsh ? dig(c, i, k - qsh) : 0;
        eus[c] = ec - qsh;
        int32_t xe[D];
        for (int k = 0; k < D; ++k) xe[k] = dig(c, c, k);
        xf<N> v0, bp, rcc, inv, bet;
        // as on the GPU: double-double FP64 scalars for P = 2, digits otherwise
        const xf<N> sig_x = xf_from_acc<N>(sacc, 2 * ec + D - 3), x0_x = xf_from_fixed<N, D>(xe, ec);
        if constexpr (P == 2) kinds[c] = xf_house_dd<N>(sig_x, x0_x, v0, bp, rcc, inv, bet);
        else kinds[c] = xf_house<N>(sig_x, x0_x, v0, bp, rcc, inv, bet);
        v0s[c] = v0;
        bps[c] = bp;
        store<P>(beta, n, c, xf_to_md<P, N>(bet));
        store<P>(col, ps, c, xf_to_md<P, N>(rcc));
        for (long i = 0; i < m; ++i) {
            if (i == c) continue;
            int32_t x[D];
            for (int k = 0; k < D; ++k) x[k] = dig(c, i, k);
            md<P> y = i < c ? xf_to_md<P, N>(xf_from_fixed<N, D>(x, ec))
                            : xf_to_md<P, N>(xf_mul<N>(xf_from_fixed<N, D>(x, eus[c]), inv));
            store<P>(col, ps, i, y);
        }
    }
    return 0;
}

extern "C" int fx_panel_replay(int p, long m, long n, double* A, double* beta) {
    if (p == 2) return panel_replay<2>(m, n, A, beta);
    if (p == 4) return panel_replay<4>(m, n, A, beta);
    return panel_replay<8>(m, n, A, beta);
}
