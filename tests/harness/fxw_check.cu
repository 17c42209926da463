// Test harness (GPU): the warp-parallel digit scalars of csrc/fxw.cuh against
// their one-thread namesakes of csrc/fx.cuh, digit for digit, on random
// inputs.  One warp per case; every lane also runs the scalar routine (the
// same inputs in every lane) and the two results must agree exactly.
#include <cstdint>

#include "../../paper_2110_08375_gb300/csrc/panel_fx.cuh"

using namespace mdls;

namespace {

__device__ uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// random sign-consistent value: digits below 2^24 with a nonzero top one,
// occasionally sparse (runs of zero or full digits exercise the carries)
template <int N>
__device__ fx::xf<N> rand_xf(uint64_t key, bool positive) {
    fx::xf<N> x;
    const uint64_t h = mix64(key);
    const int s = (positive || (h & 1)) ? 1 : -1;
    const int style = (int)((h >> 1) & 3);
    for (int k = 0; k < N; ++k) {
        const uint64_t r = mix64(key * 131 + k + 1);
        int32_t d = (int32_t)(r & fx::kMask);
        if (style == 1 && (r >> 40) % 3 == 0) d = 0;
        if (style == 2 && (r >> 40) % 3 == 0) d = (int32_t)fx::kMask;
        x.d[k] = s * d;
    }
    if (x.d[N - 1] == 0) x.d[N - 1] = s;
    x.e = (int)((h >> 8) % 41) - 20;
    return x;
}

template <int N>
__device__ bool same(const fx::xf<N>& s, const fxw::wxf& w) {
    const fx::xf<N> t = fxw::to_scalar<N>(w);
    bool ok = t.e == s.e || (fx::xf_is_zero<N>(s) && fx::xf_is_zero<N>(t));
    for (int k = 0; k < N; ++k) ok = ok && t.d[k] == s.d[k];
    return ok;
}

template <int N>
__device__ bool same_xf(const fx::xf<N>& a, const fx::xf<N>& b) {
    bool ok = a.e == b.e || (fx::xf_is_zero<N>(a) && fx::xf_is_zero<N>(b));
    for (int k = 0; k < N; ++k) ok = ok && a.d[k] == b.d[k];
    return ok;
}

template <int P>
__device__ bool same_md(const md<P>& a, const md<P>& b) {
    bool ok = true;
    for (int l = 0; l < P; ++l) ok = ok && fx::dbits(a.v[l]) == fx::dbits(b.v[l]);
    return ok;
}

// bad[op] counts the cases where op differs; ops: 0 mul, 1 add, 2 sub,
// 3 recip, 4 rsqrt, 5 house (all outputs and the kind), 6 from_double,
// 7 fixed round trip, 8 shift_bits, 9 from_acc of a wide accumulator,
// 10 from_md, 11 the panels' two-step scalars (panel_house_lead and _tail)
// against the one-thread form (xf_house_dd for P = 2, else xf_house)
constexpr int kOps = 12;

template <int P, int N, int D>
__global__ void check_kernel(int cases, uint64_t seed, int* bad) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= cases) return;  // whole warp
    const uint64_t key = seed * 1000003ULL + (uint64_t)w * 7919ULL;
    const int lane = threadIdx.x & 31;
    fx::xf<N> a = rand_xf<N>(key, false), b = rand_xf<N>(key + 1, false);
    if (w % 17 == 3) a = fx::xf_zero<N>();
    if (w % 19 == 5) b = fx::xf_zero<N>();
    if (w % 7 == 2) b.e = a.e + (int)(mix64(key + 2) % 5) - 2;  // overlapping windows, cancellation
    if (w % 11 == 4) b = fx::xf_neg<N>(a);
    const fxw::wxf wa = fxw::from_scalar<N>(a), wb = fxw::from_scalar<N>(b);
    bool ok[kOps];
    ok[0] = same<N>(fx::xf_mul<N>(a, b), fxw::mul<N>(wa, wb));
    ok[1] = same<N>(fx::xf_add<N>(a, b), fxw::add<N>(wa, wb));
    ok[2] = same<N>(fx::xf_sub<N>(a, b), fxw::sub<N>(wa, wb));
    const fx::xf<N> pa = rand_xf<N>(key + 3, true);
    const fxw::wxf wpa = fxw::from_scalar<N>(pa);
    ok[3] = same<N>(fx::xf_recip<N>(a.d[N - 1] != 0 ? a : pa),
                    fxw::recip<N>(a.d[N - 1] != 0 ? wa : wpa));
    ok[4] = same<N>(fx::xf_rsqrt<N>(pa), fxw::rsqrt<N>(wpa));
    {
        const fx::xf<N> sig = (w % 13 == 6) ? fx::xf_zero<N>() : pa;
        const fx::xf<N> x0 = b;
        fx::xf<N> v0, bp, rcc, inv, bet;
        const int kind = fx::xf_house<N>(sig, x0, v0, bp, rcc, inv, bet);
        fxw::wxf wv0, wbp, wrcc, winv, wbet;
        const int wkind = fxw::house<N>(fxw::from_scalar<N>(sig), wb, wv0, wbp, wrcc, winv, wbet);
        ok[5] = kind == wkind && same<N>(v0, wv0) && same<N>(bp, wbp) && same<N>(rcc, wrcc) &&
                same<N>(inv, winv) && same<N>(bet, wbet);
    }
    {
        const uint64_t r = mix64(key + 4);
        double v = (double)(int64_t)(r >> 11) * 0x1p-40;
        if ((r & 7) == 0) v = 0.0;
        v = ldexp(v, (int)((r >> 3) % 200) - 100);
        ok[6] = same<N>(fx::xf_from_double<N>(v), fxw::from_double<N>(v));
    }
    {
        // fixed point at a scale near a's: digits of a at scale e, back again
        const int e = a.e + (int)(mix64(key + 5) % 5) - 2;
        int32_t dd[D];
        const bool sok = fx::fixed_from_xf<N, D>(a, e, dd);
        int32_t mine;
        const bool wok = fxw::fixed_from_xf<N, D>(wa, e, mine);
        bool digits_ok = sok == wok;
        for (int k = 0; k < D; ++k) digits_ok = digits_ok && (__shfl_sync(0xffffffffu, mine, k) == dd[k]);
        ok[7] = digits_ok && same<N>(fx::xf_from_fixed<N, D>(dd, e), fxw::from_fixed<N, D>(mine, e));
    }
    {
        const int s = (int)(mix64(key + 6) % 47) - 23;
        ok[8] = same<N>(fx::xf_shift_bits<N>(a, s), fxw::shift_bits<N>(wa, s));
    }
    {
        // a wide accumulator with large mixed-sign entries (dot-product sums)
        constexpr int M = D + 3;
        int64_t c[M];
        for (int k = 0; k < M; ++k) {
            const uint64_t r = mix64(key * 3 + 100 + k);
            c[k] = (int64_t)(r >> 12) - (int64_t)(1ULL << 51);
        }
        if (w % 5 == 1) c[M - 1] = 0;
        const int64_t mine = lane < M ? c[lane] : 0;
        ok[9] = same<N>(fx::xf_from_acc<N, M>(c, -3), fxw::from_acc<N, M>(mine, -3));
    }
    {
        // P limbs, each about 2^-53 below the previous, some zero or tiny
        md<P> x;
        const uint64_t r0 = mix64(key + 7);
        double v = ldexp((double)(int64_t)(r0 >> 11) * 0x1p-53, (int)((r0 >> 3) % 120) - 60);
        for (int l = 0; l < P; ++l) {
            const uint64_t r = mix64(key * 5 + 200 + l);
            x.v[l] = (r & 15) == 0 ? 0.0 : v;
            v = v * 0x1p-53 * ((double)(int64_t)(r >> 11) * 0x1p-52) * ((r & 16) ? 1.0 : 0x1p-30);
        }
        if (w % 23 == 7) x = md_zero<P>();
        ok[10] = same<N>(fx::xf_from_md<P, N>(x), fxw::from_md<P, N>(x));
    }
    {
        // magnitudes within the double range (leading digit at 2^(24e), |e| <= 20)
        fx::xf<N> sig = (w % 13 == 6) ? fx::xf_zero<N>() : pa, x0 = b;
        if (!fx::xf_is_zero<N>(sig)) sig.e -= N - 1;
        if (!fx::xf_is_zero<N>(x0)) x0.e -= N - 1;
        fx::xf<N> v0, bp, rcc, inv, bet;
        int kind;
        if constexpr (P == 2) kind = fx::xf_house_dd<N>(sig, x0, v0, bp, rcc, inv, bet);
        else kind = fx::xf_house<N>(sig, x0, v0, bp, rcc, inv, bet);
        PanelHouse<P, N> h;
        panel_house_lead<P, N>(fxw::from_scalar<N>(sig), fxw::from_scalar<N>(x0), h);
        const bool lead_ok = h.kind == kind && same<N>(v0, h.v0) && same<N>(bp, h.bp);
        panel_house_tail<P, N>(h);
        bool tail_ok = same<N>(inv, h.inv);
        if (P == 2 && kind == 0) {
            // the panels keep R_cc and beta in limbs; the one-thread form
            // rounds them to digits
            tail_ok = tail_ok && same_xf<N>(rcc, fx::xf_from_md<P, N>(h.rcc)) &&
                      same_xf<N>(bet, fx::xf_from_md<P, N>(h.beta));
        } else {
            tail_ok = tail_ok && same_md<P>(fx::xf_to_md<P, N>(rcc), h.rcc) && same_md<P>(fx::xf_to_md<P, N>(bet), h.beta);
        }
        ok[11] = lead_ok && tail_ok;
    }
    if (lane == 0)
        for (int q = 0; q < kOps; ++q)
            if (!ok[q]) atomicAdd(bad + q, 1);
}

template <int P>
int run(int cases, uint64_t seed, int* host_bad) {
    constexpr int N = fx::Cfg<P>::N, D = fx::Cfg<P>::D;
    int* bad = nullptr;
    if (cudaMalloc(&bad, kOps * sizeof(int)) != cudaSuccess) return -1;
    cudaMemset(bad, 0, kOps * sizeof(int));
    check_kernel<P, N, D><<<(cases + 3) / 4, 128>>>(cases, seed, bad);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(bad);
        return -2;
    }
    cudaMemcpy(host_bad, bad, kOps * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(bad);
    return 0;
}

}  // namespace

extern "C" int fxw_check(int p, int cases, unsigned long long seed, int* host_bad) {
    switch (p) {
        case 2: return run<2>(cases, seed, host_bad);
        case 4: return run<4>(cases, seed, host_bad);
        case 8: return run<8>(cases, seed, host_bad);
        default: return -3;
    }
}
