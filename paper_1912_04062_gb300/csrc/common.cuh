// common.cuh -- device helpers shared by the CUDA translation units of the
// skew-symmetric eigensolver: status codes, capped waits, grid barrier,
// warp reductions.  No solver arithmetic lives here.
#pragma once
#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>

#include "../../include/skeweig.h"

#define SK_DEV __device__ __forceinline__

// Upper bound on polls of any spin wait (each poll sleeps ~64-256 ns), so a
// wait gives up after roughly one to four seconds and reports
// SKEW_ERR_DEVICE_TIMEOUT instead of hanging the GPU.
#ifndef SK_SPIN_CAP
#define SK_SPIN_CAP (1u << 24)
#endif
// Cap of the waits between CTAs under SKEW_FAULT_TINY_WAIT: a wait not
// satisfied by its second poll gives up (tests of the timeout path).
#define SK_TINY_SPIN_CAP 1u

// Device-side status word: first error wins.
SK_DEV void sk_set_error(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

SK_DEV unsigned sk_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
SK_DEV int sk_ld_acquire_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
SK_DEV void sk_st_release_s32(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
SK_DEV unsigned sk_atom_add_release(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Grid-wide barrier for cooperative launches (all CTAs co-resident).  The
// counter grows monotonically; the caller tracks its own epoch.  Returns false
// (and records SKEW_ERR_DEVICE_TIMEOUT) when the wait cap (polls) is reached or
// when another CTA already reported an error.
SK_DEV bool sk_grid_barrier(unsigned* counter, unsigned& epoch, int* status, unsigned cap = SK_SPIN_CAP) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch += 1;
        const unsigned target = epoch * gridDim.x;
        // the block's writes precede the release (bar.sync, then a gpu-scope
        // release by this thread)
        sk_atom_add_release(counter, 1u);
        int ok = 1;
        unsigned polls = 0;
        // the error word is read every 256 polls and the poll sleeps only
        // after 256 tries: a barrier completes within one L2 round trip of
        // its last arrival
        while (sk_ld_acquire(counter) < target) {
            ++polls;
            if (polls > cap || ((polls & 255u) == 0 && *(volatile int*)status != 0)) {
                ok = 0;
                break;
            }
            if (polls > 256) __nanosleep(64);
        }
        if (!ok) sk_set_error(status, SKEW_ERR_DEVICE_TIMEOUT);
        s_ok = ok;
    } else {
        epoch += 1;
    }
    __syncthreads();
    return s_ok != 0;
}

// Wait until *flag >= want (acquire).  Thread 0 polls; the block synchronises.
SK_DEV bool sk_wait_flag_geq(const int* flag, int want, int* status) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned polls = 0;
        while (sk_ld_acquire_s32(flag) < want) {
            if (++polls > SK_SPIN_CAP || *(volatile int*)status != 0) {
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        if (!ok) sk_set_error(status, SKEW_ERR_DEVICE_TIMEOUT);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
SK_DEV T sk_warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of one value per thread (blockDim.x <= 1024).  All threads
// receive the result.  scratch must hold 32 elements.
template <typename T>
SK_DEV T sk_block_sum(T v, T* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = sk_warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    T r = (threadIdx.x < nw) ? scratch[threadIdx.x] : T(0);
    if (warp == 0) r = sk_warp_sum(r);
    if (threadIdx.x == 0) scratch[0] = r;
    __syncthreads();
    r = scratch[0];
    __syncthreads();
    return r;
}

SK_DEV double sk_ldcg(const double* p) { return __ldcg(p); }
