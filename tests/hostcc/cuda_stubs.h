// Host-compiler stand-ins for the CUDA device builtins the library uses, so
// that g++ can type-check its device code (-Wconversion) and run its pure
// integer helpers on the host.  Builtins whose value matters to those helpers
// are defined by their mathematics; the others are inert.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <algorithm>

extern const uint3 threadIdx, blockIdx;
extern const dim3 blockDim, gridDim;
static const int warpSize = 32;

inline void __syncthreads() {}
inline void __syncwarp(unsigned = 0xffffffffu) {}
inline void __threadfence() {}
inline void __nanosleep(unsigned) {}
template <class T> T __shfl_sync(unsigned, T v, int, int = 32) { return v; }
template <class T> T __shfl_xor_sync(unsigned, T v, int, int = 32) { return v; }
template <class T> T __shfl_up_sync(unsigned, T v, unsigned, int = 32) { return v; }
template <class T> T __shfl_down_sync(unsigned, T v, unsigned, int = 32) { return v; }
inline unsigned __ballot_sync(unsigned, int) { return 0; }
inline int __any_sync(unsigned, int) { return 0; }
inline int __all_sync(unsigned, int) { return 0; }
template <class T> unsigned __match_any_sync(unsigned, T) { return 0; }
inline int __reduce_max_sync(unsigned, int v) { return v; }
inline unsigned __reduce_max_sync(unsigned, unsigned v) { return v; }
inline int __reduce_add_sync(unsigned, int v) { return v; }
inline unsigned __reduce_add_sync(unsigned, unsigned v) { return v; }
inline int __popc(unsigned) { return 0; }
inline int __popcll(unsigned long long) { return 0; }
inline int __ffs(int) { return 0; }
inline int __clz(int) { return 0; }
inline int __clzll(long long) { return 0; }
// the high 64 bits of the 128-bit product (its definition)
inline unsigned long long __umul64hi(unsigned long long a, unsigned long long b) {
    return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
inline double __ull2double_rn(unsigned long long x) { return (double)x; }
inline size_t __cvta_generic_to_shared(const void *) { return 0; }
template <class T> T __ldg(const T *p) { return *p; }
template <class T> T __ldcg(const T *p) { return *p; }
template <class T> void __stcg(T *p, T v) { *p = v; }

inline int atomicAdd(int *, int v) { return v; }
inline unsigned atomicAdd(unsigned *, unsigned v) { return v; }
inline unsigned long long atomicAdd(unsigned long long *, unsigned long long v) { return v; }
inline float atomicAdd(float *, float v) { return v; }
inline double atomicAdd(double *, double v) { return v; }
inline int atomicMax(int *, int v) { return v; }
inline unsigned atomicMax(unsigned *, unsigned v) { return v; }
inline long long atomicMax(long long *, long long v) { return v; }
inline unsigned long long atomicMax(unsigned long long *, unsigned long long v) { return v; }
inline int atomicMin(int *, int v) { return v; }
inline long long atomicMin(long long *, long long v) { return v; }
inline int atomicOr(int *, int v) { return v; }
inline unsigned atomicOr(unsigned *, unsigned v) { return v; }
inline unsigned long long atomicOr(unsigned long long *, unsigned long long v) { return v; }
inline int atomicAnd(int *, int v) { return v; }
inline unsigned atomicAnd(unsigned *, unsigned v) { return v; }
inline int atomicExch(int *, int v) { return v; }
inline unsigned atomicExch(unsigned *, unsigned v) { return v; }
inline unsigned long long atomicExch(unsigned long long *, unsigned long long v) { return v; }
inline int atomicCAS(int *, int, int v) { return v; }
inline unsigned atomicCAS(unsigned *, unsigned, unsigned v) { return v; }
inline unsigned long long atomicCAS(unsigned long long *, unsigned long long, unsigned long long v) { return v; }

// CUDA's integer min/max overloads
inline int min(int a, int b) { return a < b ? a : b; }
inline unsigned min(unsigned a, unsigned b) { return a < b ? a : b; }
inline long long min(long long a, long long b) { return a < b ? a : b; }
inline long min(long a, long b) { return a < b ? a : b; }
inline unsigned long long min(unsigned long long a, unsigned long long b) { return a < b ? a : b; }
inline unsigned long min(unsigned long a, unsigned long b) { return a < b ? a : b; }
inline long long min(int a, long long b) { return a < b ? a : b; }
inline long long min(long long a, int b) { return a < b ? a : b; }
inline long min(int a, long b) { return a < b ? a : b; }
inline long min(long a, int b) { return a < b ? a : b; }
inline int max(int a, int b) { return a > b ? a : b; }
inline unsigned max(unsigned a, unsigned b) { return a > b ? a : b; }
inline long long max(long long a, long long b) { return a > b ? a : b; }
inline long max(long a, long b) { return a > b ? a : b; }
inline unsigned long long max(unsigned long long a, unsigned long long b) { return a > b ? a : b; }
inline unsigned long max(unsigned long a, unsigned long b) { return a > b ? a : b; }
inline long long max(int a, long long b) { return a > b ? a : b; }
inline long long max(long long a, int b) { return a > b ? a : b; }
inline long max(int a, long b) { return a > b ? a : b; }
inline long max(long a, int b) { return a > b ? a : b; }
#ifndef __launch_bounds__
#define __launch_bounds__(...)
#endif
