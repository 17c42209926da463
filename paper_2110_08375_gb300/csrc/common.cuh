// Shared device definitions: limb-planar matrix views and the workspace
// header (device status word, failure flag of the bounded waits).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mdls.h"
#include "md.cuh"

namespace mdls {

#define DEV_INLINE __device__ __forceinline__

// Limb-planar storage ("staggered" storage of the paper's Section 2): limb l
// of entry (i, j) sits at ptr[l * ps + j * ld + i].
struct Dense {
    double* ptr;
    int64_t ld, ps;
};

template <int P>
DEV_INLINE md<P> ld_md(const double* __restrict__ ptr, int64_t ps, int64_t off) {
    md<P> r;
#pragma unroll
    for (int l = 0; l < P; ++l) r.v[l] = ptr[l * ps + off];
    return r;
}

template <int P>
DEV_INLINE void st_md(double* __restrict__ ptr, int64_t ps, int64_t off, const md<P>& x) {
#pragma unroll
    for (int l = 0; l < P; ++l) ptr[l * ps + off] = x.v[l];
}

// Operand views for the md GEMM.  get(i, k, l) returns limb l of element
// (i, k) of the operand as the GEMM sees it.
// kRowContig: consecutive i are consecutive in memory (column-major rows).
// Known zero structure, used by the products to skip k ranges that only meet
// zeros: kZeroKBelowI (element (i, k) = 0 for k < i, upper triangular) and
// kZeroKAboveI (element (i, k) = 0 for k > i, lower triangular / trapezoid).
struct ViewDense {      // X(i, k)
    static constexpr bool kRowContig = true;
    static constexpr bool kZeroKBelowI = false, kZeroKAboveI = false;
    const double* ptr;
    int64_t ld, ps;
    DEV_INLINE double get(int64_t i, int64_t k, int l) const { return ptr[l * ps + k * ld + i]; }
};
struct ViewDenseT {     // X(k, i): the transpose
    static constexpr bool kRowContig = false;
    static constexpr bool kZeroKBelowI = false, kZeroKAboveI = false;
    const double* ptr;
    int64_t ld, ps;
    DEV_INLINE double get(int64_t i, int64_t k, int l) const { return ptr[l * ps + i * ld + k]; }
};
// Unit lower trapezoid Y of Householder vectors stored below the diagonal:
// Y(i, k) = 0 for i < k, 1 for i == k, stored value for i > k.
struct ViewTrap {
    static constexpr bool kRowContig = true;
    static constexpr bool kZeroKBelowI = false, kZeroKAboveI = true;
    const double* ptr;  // points at the panel's (0, 0)
    int64_t ld, ps;
    DEV_INLINE double get(int64_t i, int64_t k, int l) const {
        if (i > k) return ptr[l * ps + k * ld + i];
        return (i == k && l == 0) ? 1.0 : 0.0;
    }
};
struct ViewTrapT {      // Y^T
    static constexpr bool kRowContig = false;
    static constexpr bool kZeroKBelowI = true, kZeroKAboveI = false;
    const double* ptr;
    int64_t ld, ps;
    DEV_INLINE double get(int64_t i, int64_t k, int l) const {
        if (k > i) return ptr[l * ps + i * ld + k];
        return (k == i && l == 0) ? 1.0 : 0.0;
    }
};
// Upper triangular operand (entries below the diagonal read as zero).
struct ViewUpper {
    static constexpr bool kRowContig = true;
    static constexpr bool kZeroKBelowI = true, kZeroKAboveI = false;
    const double* ptr;
    int64_t ld, ps;
    DEV_INLINE double get(int64_t i, int64_t k, int l) const {
        return (i <= k) ? ptr[l * ps + k * ld + i] : 0.0;
    }
};
// Transpose of an upper triangular matrix X: element (i, k) = X(k, i), zero
// for k > i.
struct ViewUpperT {
    static constexpr bool kRowContig = false;
    static constexpr bool kZeroKBelowI = false, kZeroKAboveI = true;
    const double* ptr;
    int64_t ld, ps;
    DEV_INLINE double get(int64_t i, int64_t k, int l) const {
        return (k <= i) ? ptr[l * ps + i * ld + k] : 0.0;
    }
};

// ----------------------------------------------------------------------------
// Workspace header: the status word and the failure flag of the bounded waits
// live at the start of every workspace the caller hands in.
// ----------------------------------------------------------------------------
struct WsHeader {
    int status;                  // first error seen on the device (0 = none)
    int pad0;
    unsigned long long wait_ns;  // limit of every bounded wait, ns (0 = the 2 s default)
    int bar_error;               // set by a bounded wait that gave up: later waits fail fast
    int pad2[59];                // header is 256 bytes
};
static_assert(sizeof(WsHeader) == 256, "workspace header must be 256 bytes");

DEV_INLINE void set_status(int* status, int code) { atomicCAS(status, 0, code); }

}  // namespace mdls
