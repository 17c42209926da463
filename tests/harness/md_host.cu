// Test harness: the device md arithmetic of csrc/md.cuh compiled for the host,
// exposed with a C interface so the tests can compare it with the oracle on
// the CPU.  Built with -ffp-contract=off so that the host compiler keeps every
// operation as written.
#include "../../paper_2110_08375_gb300/csrc/md.cuh"

using namespace mdls;

template <int P>
static void run(int op, long n, const double* a, const double* b, double* c) {
    for (long i = 0; i < n; ++i) {
        md<P> x, y, z;
        for (int l = 0; l < P; ++l) {
            x.v[l] = a[l * n + i];
            y.v[l] = b[l * n + i];
            z.v[l] = c[l * n + i];
        }
        md<P> r;
        switch (op) {
            case 0: r = md_add<P>(x, y); break;
            case 1: r = md_sub<P>(x, y); break;
            case 2: r = md_mul<P>(x, y); break;
            case 3: r = md_div<P>(x, y); break;
            case 4: r = md_fma<P>(z, x, y); break;
            default: r = md_sqrt<P>(x); break;
        }
        for (int l = 0; l < P; ++l) c[l * n + i] = r.v[l];
    }
}

extern "C" void md_host_op(int p, int op, long n, const double* a, const double* b, double* c) {
    if (p == 2) run<2>(op, n, a, b, c);
    else if (p == 4) run<4>(op, n, a, b, c);
    else run<8>(op, n, a, b, c);
}

// two_sum in its two forms: 0 the integer error (two_sum_int), 1 Fast2Sum
// after the integer ordering (two_sum_fast)
extern "C" void md_host_two_sum(int form, long n, const double* a, const double* b, double* s, double* e) {
    for (long i = 0; i < n; ++i) {
        if (form == 0) two_sum_int(a[i], b[i], s[i], e[i]);
        else two_sum_fast(a[i], b[i], s[i], e[i]);
    }
}
