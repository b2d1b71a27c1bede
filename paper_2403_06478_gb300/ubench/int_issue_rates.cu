// Integer issue-rate microbenchmark (not part of the library): ops per clock per
// SM of the candidate DP operations, each in 8 independent chains, 1 block of
// 512 or 1024 threads per SM, cycles from clock64().  Used to derive the
// integer-issue roofline of the alignment kernels.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define ITERS 4096
#define CHAINS 8

template <int OP>
__device__ __forceinline__ int op(int a, int b, int c) {
    if constexpr (OP == 0) return a + b;                          // IADD
    if constexpr (OP == 1) return max(a, b);                      // IMNMX
    if constexpr (OP == 2) return __viaddmax_s32(a, b, c);        // DPX add-max
    if constexpr (OP == 3) return __vimax3_s32(a, b, c);          // DPX 3-way max
    if constexpr (OP == 4) return (int)__viaddmax_s16x2((unsigned)a, (unsigned)b, (unsigned)c);
    if constexpr (OP == 5) return (int)__vimax3_s16x2((unsigned)a, (unsigned)b, (unsigned)c);
    if constexpr (OP == 6) return (int)__vmaxs2((unsigned)a, (unsigned)b);
    if constexpr (OP == 7) return (int)__vadd2((unsigned)a, (unsigned)b);
    if constexpr (OP == 8) return (a ^ b) & c;                    // LOP3
    if constexpr (OP == 9) return (a & 0x40) ? b : c;             // test + select
    if constexpr (OP == 10) return __viaddmin_s32(a, b, c);
    if constexpr (OP == 11) return a + b + c;                     // IADD3
    if constexpr (OP == 12) return (int)__viaddmax_u16x2((unsigned)a, (unsigned)b, (unsigned)c);
    if constexpr (OP == 13) return max(max(a, b), c);             // two IMNMX or one 3-input
    if constexpr (OP == 14) return __shfl_xor_sync(0xffffffffu, a, 1) + b;
    if constexpr (OP == 15) return a * b + c;                     // IMAD
    if constexpr (OP == 16) return (int)__vmaxu2((unsigned)a, (unsigned)b);
    if constexpr (OP == 17) {                                     // prmt sign-replicate
        unsigned d;
        asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(0xbb99));
        return (int)d;
    }
    if constexpr (OP == 18) return (int)__viaddmin_u16x2((unsigned)a, (unsigned)b, (unsigned)c);
    if constexpr (OP == 19) return (int)__vminu2((unsigned)a, (unsigned)b);
    if constexpr (OP == 20) return (a << 3) + b;                  // shift + add (LEA)
    if constexpr (OP == 21) {                                     // one packed bulk cell
        unsigned H = __viaddmax_u16x2((unsigned)a, (unsigned)b, (unsigned)c);
        H = __vmaxu2(H, (unsigned)b ^ 7u);
        H = __vmaxu2(H, __vmaxu2((unsigned)c ^ 3u, (unsigned)b ^ 5u));
        unsigned hoe = H - 0x00060006u;
        unsigned e1 = __vmaxu2((unsigned)b - 0x00020002u, hoe);
        unsigned f1 = __vmaxu2((unsigned)c - 0x00020002u, hoe);
        unsigned hoe2 = hoe - 0x00140014u;
        unsigned e2 = __vmaxu2((unsigned)b - 0x00010001u, hoe2);
        unsigned f2 = __vmaxu2((unsigned)c - 0x00010001u, hoe2);
        return (int)(e1 ^ f1 ^ e2 ^ f2 ^ H);
    }
    return a;
}

template <int OP>
__global__ void bench(int *out, long long *cycles, int seed) {
    int acc[CHAINS];
    int b = seed * 3 + threadIdx.x, c = seed ^ 0x5a5a5a;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) acc[i] = seed + i * 7 + threadIdx.x;
    __syncthreads();
    long long t0 = clock64();
    for (int it = 0; it < ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) acc[i] = op<OP>(acc[i], b, c);
        b ^= it;   // keep operands live
    }
    __syncthreads();
    long long t1 = clock64();
    int s = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s ^= acc[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int OP>
void run(const char *name, int nsm, int threads, int *d_out, long long *d_cyc) {
    bench<OP><<<nsm, threads>>>(d_out, d_cyc, 1);
    cudaDeviceSynchronize();
    bench<OP><<<nsm, threads>>>(d_out, d_cyc, 2);
    cudaDeviceSynchronize();
    long long h[1024];
    cudaMemcpy(h, d_cyc, nsm * sizeof(long long), cudaMemcpyDeviceToHost);
    double mean = 0;
    for (int i = 0; i < nsm; ++i) mean += h[i];
    mean /= nsm;
    double ops = (double)threads * ITERS * CHAINS;
    printf("%-16s %7.1f ops/clk/SM (threads %d)\n", name, ops / mean, threads);
}

int main() {
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, 0);
    int nsm = p.multiProcessorCount;
    printf("%s, %d SMs, cc %d.%d\n", p.name, nsm, p.major, p.minor);
    int *d_out;
    long long *d_cyc;
    cudaMalloc(&d_out, nsm * 1024 * sizeof(int));
    cudaMalloc(&d_cyc, nsm * sizeof(long long));
    for (int threads : {512, 1024}) {
        run<0>("iadd", nsm, threads, d_out, d_cyc);
        run<11>("iadd3", nsm, threads, d_out, d_cyc);
        run<1>("imax", nsm, threads, d_out, d_cyc);
        run<13>("max(max)", nsm, threads, d_out, d_cyc);
        run<2>("viaddmax_s32", nsm, threads, d_out, d_cyc);
        run<10>("viaddmin_s32", nsm, threads, d_out, d_cyc);
        run<3>("vimax3_s32", nsm, threads, d_out, d_cyc);
        run<4>("viaddmax_s16x2", nsm, threads, d_out, d_cyc);
        run<12>("viaddmax_u16x2", nsm, threads, d_out, d_cyc);
        run<5>("vimax3_s16x2", nsm, threads, d_out, d_cyc);
        run<6>("vmaxs2", nsm, threads, d_out, d_cyc);
        run<7>("vadd2", nsm, threads, d_out, d_cyc);
        run<8>("lop3", nsm, threads, d_out, d_cyc);
        run<9>("test+sel", nsm, threads, d_out, d_cyc);
        run<15>("imad", nsm, threads, d_out, d_cyc);
        run<14>("shfl+add", nsm, threads, d_out, d_cyc);
        run<16>("vmaxu2", nsm, threads, d_out, d_cyc);
        run<17>("prmt", nsm, threads, d_out, d_cyc);
        run<18>("viaddmin_u16x2", nsm, threads, d_out, d_cyc);
        run<19>("vminu2", nsm, threads, d_out, d_cyc);
        run<20>("shl+add", nsm, threads, d_out, d_cyc);
        run<21>("packed cell (x1)", nsm, threads, d_out, d_cyc);
    }
    cudaError_t e = cudaGetLastError();
    printf("status: %s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
