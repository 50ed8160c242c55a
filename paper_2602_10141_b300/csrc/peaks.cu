// Issue-rate probes for the pipes the Ryser kernels use.  They give the
// roofline denominators that the measured HBM copy and bf16 GEMM peaks do not
// cover: FP64 (f64 / complex128 walks) and 32-bit integer (F_p walk).
//
// Each thread runs 8 independent dependency chains of one operation for
// `iters` iterations; the operations per second are blocks*threads*iters*8
// divided by the CUDA-event time of the launch.  Kinds:
//   0 fma.rn.f64   1 add.rn.f64   2 mul.rn.f64   3 fma.rn.f32
//   4 mad.lo.u32   5 mul.wide.u32 6 mul.hi.u32   7 add.u32   8 min.u32
//   9 one F_p unit (modular add + Montgomery multiply, as in the F_p walk)
//  10 one float64 unit (add + multiply)  11 one complex128 unit (2 adds + complex multiply)
//  12 clz.b64   13 clz.b32   14 one real integer-mantissa factor (x64_mul)
//  15 one complex integer-mantissa factor (x64c_mul)
//  16 one real integer-mantissa term: int64 row-sum update + chain factor (x64_mul_row)
//  17 one complex integer-mantissa term: two int64 updates + chain factor (x64c_mul_row)
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "x64_arith.cuh"

namespace permx {

template <int KIND>
__global__ void peak_kernel(int iters, uint32_t seed, unsigned long long* sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    double d[8], e = 0.9999999 + 1e-9 * (seed & 7), f = 1e-7;
    float fl[8];
    uint32_t u[8], v = seed | 1u, w = tid ^ seed;
    uint32_t t[8];
    double2 c[8], cr[8];
    const uint32_t p = 2147483629u, pinv = 1681680005u;   // any odd p and its inverse mod 2^32
    // kinds 16 / 17: staged-size row sums (|Re| + |Im| < 2^62) and normalised mantissas
    int64_t Rr[8], Ri[8];
    XReal xr[8];
    XCplx xc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        Rr[k] = 0x2d00000000000000ll + ((int64_t)(tid + k) << 20);
        Ri[k] = 0x1200000000000000ll - ((int64_t)(3 * tid + k) << 18);
        xr[k] = XReal{0x3000000000000000ll + k, 0};
        xc[k] = XCplx{0x1800000000000000ll + k, 0x0c00000000000000ll - k, 0};
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        d[k] = 1.0 + k * 1e-3 + tid * 1e-9;
        fl[k] = 1.0f + k * 1e-3f;
        u[k] = tid * 2654435761u + k;
        t[k] = (tid + k) % p;
        c[k] = make_double2(0.5 + k * 1e-3, 0.25);
        cr[k] = make_double2(0.75, -0.5 + k * 1e-3);
    }
    for (int it = 0; it < iters; ++it) {
        const int64_t dv = (it & 1) ? (int64_t)v << 24 : -((int64_t)v << 24);   // row sums stay in range
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (KIND == 16) {
                Rr[k] += dv;
                xr[k] = x64_mul_row(xr[k], Rr[k]);
            }
            if (KIND == 17) {
                Rr[k] += dv;
                Ri[k] -= dv;
                xc[k] = x64c_mul_row(xc[k], Rr[k], Ri[k]);
            }
            if (KIND == 0) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d[k]) : "d"(e), "d"(f));
            if (KIND == 1) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(d[k]) : "d"(f));
            if (KIND == 2) asm volatile("mul.rn.f64 %0, %0, %1;" : "+d"(d[k]) : "d"(e));
            if (KIND == 3) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(fl[k]) : "f"((float)e), "f"((float)f));
            if (KIND == 4) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(u[k]) : "r"(v), "r"(w));
            if (KIND == 5) {
                uint64_t r;
                asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(r) : "r"(u[k]), "r"(v));
                u[k] = (uint32_t)r ^ (uint32_t)(r >> 32);
            }
            if (KIND == 6) asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(u[k]) : "r"(v));
            if (KIND == 7) asm volatile("add.u32 %0, %0, %1;" : "+r"(u[k]) : "r"(v));
            if (KIND == 8) asm volatile("min.u32 %0, %0, %1;" : "+r"(u[k]) : "r"(w));
            if (KIND == 9) {
                uint32_t s = u[k] % p + v % p;            // hoisted by the compiler: modular add below
                uint32_t r = t[k] + (s & 0x3fffffffu);
                r = min(r, r - p);
                uint64_t T = (uint64_t)t[k] * r;
                uint32_t m = (uint32_t)T * pinv;
                uint32_t x = (uint32_t)(T >> 32) - __umulhi(m, p);
                t[k] = min(x, x + p);
            }
            if (KIND == 10) {
                d[k] = d[k] + f;
                d[k] = d[k] * e;
            }
            if (KIND == 12) {
                uint32_t z;
                asm volatile("clz.b64 %0, %1;" : "=r"(z) : "l"((unsigned long long)u[k] << 20 | t[k]));
                u[k] += z;
            }
            if (KIND == 13) asm volatile("clz.b32 %0, %0;" : "+r"(u[k]));
            if (KIND == 14) {
                XReal x{(int64_t)(((uint64_t)u[k] << 29) | 0x2000000000000000ull), 0};
                x = x64_mul(x, (int64_t)((uint64_t)v << 28) + t[k], 0);
                u[k] = (uint32_t)x.m ^ (uint32_t)x.e;
            }
            if (KIND == 15) {
                XCplx x{(int64_t)(((uint64_t)u[k] << 28) | 0x1000000000000000ull), (int64_t)t[k] << 30, 0};
                x = x64c_mul(x, (int64_t)((uint64_t)v << 28) + t[k], (int64_t)w << 27, 0);
                u[k] = (uint32_t)x.re ^ (uint32_t)x.im ^ (uint32_t)x.e;
            }
            if (KIND == 11) {
                cr[k].x += f;
                cr[k].y -= f;
                c[k] = make_double2(fma(c[k].x, cr[k].x, -c[k].y * cr[k].y), fma(c[k].x, cr[k].y, c[k].y * cr[k].x));
            }
        }
    }
    unsigned long long acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        acc += (unsigned long long)(d[k] * 1e6) + (unsigned long long)(fl[k] * 1e3f) + u[k] + t[k] +
               (unsigned long long)(c[k].x * 1e6) + (unsigned long long)(xr[k].m ^ xr[k].e) +
               (unsigned long long)(xc[k].re ^ xc[k].im ^ xc[k].e);
    if (acc == 0x123456789ull) *sink = acc;   // practically never; keeps the chains live
}

template <int KIND>
static cudaError_t run_probe(int blocks, int threads, int iters, unsigned long long* sink, float* ms) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    peak_kernel<KIND><<<blocks, threads>>>(iters / 8 + 1, 7u, sink);   // warm-up
    cudaEventRecord(a);
    peak_kernel<KIND><<<blocks, threads>>>(iters, 7u, sink);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

}  // namespace permx

using namespace permx;

extern "C" int permx_peak_probe(int kind, int blocks, int threads, int iters, double* ops_per_s, double* ms_out) {
    if (!ops_per_s || blocks < 1 || threads < 32 || threads > 1024 || iters < 1) return fail(PERMX_EINVAL, "bad arguments");
    if (kind < 0 || kind > 17) return fail(PERMX_EINVAL, "bad probe kind");
    unsigned long long* sink = nullptr;
    PERMX_CUDA(cudaMalloc(&sink, sizeof(unsigned long long)));
    float ms = 0.f;
    cudaError_t e = cudaErrorInvalidValue;
    switch (kind) {
        case 0: e = run_probe<0>(blocks, threads, iters, sink, &ms); break;
        case 1: e = run_probe<1>(blocks, threads, iters, sink, &ms); break;
        case 2: e = run_probe<2>(blocks, threads, iters, sink, &ms); break;
        case 3: e = run_probe<3>(blocks, threads, iters, sink, &ms); break;
        case 4: e = run_probe<4>(blocks, threads, iters, sink, &ms); break;
        case 5: e = run_probe<5>(blocks, threads, iters, sink, &ms); break;
        case 6: e = run_probe<6>(blocks, threads, iters, sink, &ms); break;
        case 7: e = run_probe<7>(blocks, threads, iters, sink, &ms); break;
        case 8: e = run_probe<8>(blocks, threads, iters, sink, &ms); break;
        case 9: e = run_probe<9>(blocks, threads, iters, sink, &ms); break;
        case 10: e = run_probe<10>(blocks, threads, iters, sink, &ms); break;
        case 11: e = run_probe<11>(blocks, threads, iters, sink, &ms); break;
        case 12: e = run_probe<12>(blocks, threads, iters, sink, &ms); break;
        case 13: e = run_probe<13>(blocks, threads, iters, sink, &ms); break;
        case 14: e = run_probe<14>(blocks, threads, iters, sink, &ms); break;
        case 15: e = run_probe<15>(blocks, threads, iters, sink, &ms); break;
        case 16: e = run_probe<16>(blocks, threads, iters, sink, &ms); break;
        case 17: e = run_probe<17>(blocks, threads, iters, sink, &ms); break;
        default: break;
    }
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "peak probe");
    *ops_per_s = (double)blocks * threads * (double)iters * 8.0 / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return PERMX_OK;
}
