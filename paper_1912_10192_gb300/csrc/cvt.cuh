// cvt.cuh -- binary32 <-> binary64 conversions on the integer pipe.
//
// The hardware conversions issue on the FP64 pipe, the scarce unit of this
// chip (its measured FMA rate is about 1.7 operations per SM per cycle,
// against 128 for FP32): in the FP64-pipe-bound mixed-precision cell update
// every value narrowed to FP32 or widened back costs as much as a DFMA.
// These functions do the same conversions with 32-bit integer operations on
// the bit patterns of the IEEE 754 binary32 and binary64 formats (1 sign bit;
// 8 / 11 exponent bits, biases 127 / 1023; 23 / 52 fraction bits): exact
// widening, and narrowing that rounds to nearest with ties to even (IEEE 754
// roundTiesToEven), both equal bit for bit to the hardware conversions
// (checked over every binary32 value and the rounding neighbourhoods by
// hamr_check_conversions; NaNs stay NaNs). The narrowing of values whose
// result is not a normal binary32 number (zero excepted), and of infinities
// and NaNs, takes the hardware conversion, out of line. They cost about ten
// integer instructions each, so kernels that are bound by issue or memory
// rather than by the FP64 pipe (face fluxes, EMFs, the FP32 copy of the state)
// keep the hardware conversions (measured: those kernels got slower, the cell
// update 4% faster).
#pragma once

namespace hamr {

// the hardware narrowing of the rare cases, kept out of line: a call is a real branch, where an
// inlined conversion would be predicated and still issue to the FP64 pipe in every warp
static __device__ __noinline__ float narrow_hw(double x) { return __double2float_rn(x); }

// binary32 -> binary64, exact, without branches or calls (the selects below are all integer): a
// normal value's exponent rebiased by 1023 - 127 = 896 and its 23 fraction bits moved to the top of
// the 52; a subnormal one normalised by its leading zeros (value a 2^-149 with the leading one at bit
// 31 - lz: exponent 905 - lz); zero; infinity and NaN (all-ones exponent, the fraction kept, a NaN
// made quiet)
__device__ __forceinline__ double widen(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned a = b & 0x7fffffffu;
    const unsigned lz = __clz(a);
    const unsigned ms = (a << ((lz - 8u) & 31u)) & 0x007fffffu;
    unsigned hi, lo;
    if (a - 0x00800000u < 0x7f000000u) {  // normal: biased exponent 1..254
        hi = (a >> 3) + 0x38000000u;
        lo = b << 29;
    } else if (a == 0u) {
        hi = 0u;
        lo = 0u;
    } else if (a < 0x00800000u) {  // subnormal
        hi = ((905u - lz) << 20) | (ms >> 3);
        lo = ms << 29;
    } else {  // infinity, NaN
        const unsigned f = a & 0x007fffffu;
        hi = 0x7ff00000u | (f >> 3) | (f ? 0x00080000u : 0u);
        lo = f << 29;
    }
    return __hiloint2double((int)((b & 0x80000000u) | hi), (int)lo);
}

// binary64 -> binary32, round to nearest, ties to even: the top 23 of the 52
// fraction bits, plus one where the 29 dropped bits exceed half a unit or equal
// it with an odd result (a carry into the exponent is the correct rounding,
// up to infinity)
__device__ __forceinline__ float narrow(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned a = hi & 0x7fffffffu;
    if (a - 0x38100000u < 0x0fe00000u) {  // binary64 exponent 897..1150: a normal binary32 before rounding
        unsigned f = ((a - 0x38000000u) << 3) | (lo >> 29);
        const unsigned r = lo & 0x1fffffffu;
        f += (r > 0x10000000u || (r == 0x10000000u && (f & 1u))) ? 1u : 0u;
        return __uint_as_float((hi & 0x80000000u) | f);
    }
    if ((a | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
    return narrow_hw(x);
}

// T from an FP64 value, FP64 from a T (the identity for T = double)
template <typename T>
__device__ __forceinline__ T to_t(double x) {
    if constexpr (sizeof(T) == sizeof(float))
        return narrow(x);
    else
        return x;
}

template <typename T>
__device__ __forceinline__ double to_d(T x) {
    if constexpr (sizeof(T) == sizeof(float))
        return widen(x);
    else
        return x;
}

}  // namespace hamr
