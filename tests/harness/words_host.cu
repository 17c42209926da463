// Test harness: the multiword-integer sums of the split products
// (csrc/words.cuh) compiled for the host with a C interface, so that the
// tests can compare them with exact integer arithmetic.
#include <stdint.h>

#include "../../paper_2110_08375_gb300/csrc/words.cuh"

using namespace mdls;

template <int P, int GW>
static void run(const int64_t* W, int e0, int negate, const double* c, double* out) {
    int64_t w[GW];
    for (int g = 0; g < GW; ++g) w[g] = negate ? -W[g] : W[g];  // the product is negated, not the addend
    if (c) {
        md<P> x;
        for (int l = 0; l < P; ++l) x.v[l] = c[l];
        words::add_md<GW, P>(w, x, e0);
    }
    const md<P> r = words::to_md<P, GW>(w, e0, false);
    for (int l = 0; l < P; ++l) out[l] = r.v[l];
}

// words: GW int64 words (GW = 7, 10, 17 for P = 2, 4, 8); c: P limbs or NULL.
// Returns 0, or -1 for an unsupported (P, GW).
extern "C" int words_host_to_md(int P, int GW, const int64_t* W, int e0, int negate, const double* c,
                                double* out) {
    if (P == 2 && GW == 7) run<2, 7>(W, e0, negate, c, out);
    else if (P == 4 && GW == 10) run<4, 10>(W, e0, negate, c, out);
    else if (P == 8 && GW == 17) run<8, 17>(W, e0, negate, c, out);
    else return -1;
    return 0;
}
