// ADD / ADD-S pose errors (the accuracy measure of Sec. VI): the mean over a
// mesh's vertices x of || A x - B x || (ADD) or of the distance from A x to
// the closest B y (ADD-S, for symmetric objects).  One block per pose pair;
// B's transformed vertices are staged through shared memory in tiles.
#include "perch_internal.cuh"

namespace perch {

namespace {

constexpr int kAddThreads = 256;
constexpr int kAddTile = 1024;      // B-transformed vertices per shared-memory tile
constexpr int kAddPer = 4;          // A-transformed vertices per thread per pass

__device__ __forceinline__ float3 xform(const float* P, float4 v)
{
    return make_float3(P[0] * v.x + P[1] * v.y + P[2] * v.z + P[3],
                       P[4] * v.x + P[5] * v.y + P[6] * v.z + P[7],
                       P[8] * v.x + P[9] * v.y + P[10] * v.z + P[11]);
}

__global__ void __launch_bounds__(kAddThreads) k_add_s(const float4* verts, int nv, const float* A_all,
                                                      const float* B_all, long long n, int symmetric,
                                                      double* out)
{
    __shared__ float3 tile[kAddTile];
    __shared__ float sA[12], sB[12];
    __shared__ double red[kAddThreads / 32];
    for (long long q = blockIdx.x; q < n; q += gridDim.x) {
        if (threadIdx.x < 12) {
            sA[threadIdx.x] = A_all[q * 12 + threadIdx.x];
            sB[threadIdx.x] = B_all[q * 12 + threadIdx.x];
        }
        __syncthreads();
        double acc = 0.0;
        for (int base = 0; base < nv; base += kAddThreads * kAddPer) {
            float3 pa[kAddPer];
            float best[kAddPer];
#pragma unroll
            for (int k = 0; k < kAddPer; ++k) {
                const int i = base + k * kAddThreads + threadIdx.x;
                pa[k] = i < nv ? xform(sA, verts[i]) : make_float3(0.f, 0.f, 0.f);
                best[k] = 3.0e38f;
                if (!symmetric && i < nv) {
                    const float3 pb = xform(sB, verts[i]);
                    const float dx = pa[k].x - pb.x, dy = pa[k].y - pb.y, dz = pa[k].z - pb.z;
                    best[k] = dx * dx + dy * dy + dz * dz;
                }
            }
            if (symmetric) {
                for (int t0 = 0; t0 < nv; t0 += kAddTile) {
                    const int tn = min(kAddTile, nv - t0);
                    __syncthreads();
                    for (int j = threadIdx.x; j < tn; j += kAddThreads) tile[j] = xform(sB, verts[t0 + j]);
                    __syncthreads();
                    for (int j = 0; j < tn; ++j) {
                        const float3 pb = tile[j];
#pragma unroll
                        for (int k = 0; k < kAddPer; ++k) {
                            const float dx = pa[k].x - pb.x, dy = pa[k].y - pb.y, dz = pa[k].z - pb.z;
                            best[k] = fminf(best[k], dx * dx + dy * dy + dz * dz);
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kAddPer; ++k)
                if (base + k * kAddThreads + (int)threadIdx.x < nv) acc += sqrt((double)best[k]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < kAddThreads / 32; ++w) s += red[w];
            out[q] = s / (double)nv;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_add_s(const float4* verts, int n_verts, const float* poses, const float* poses_true,
                         long long n, int symmetric, double* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (n_verts < 1) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)(n < 65535 ? n : 65535);
    k_add_s<<<grid, kAddThreads, 0, s>>>(verts, n_verts, poses, poses_true, n, symmetric, out);
    return cudaGetLastError();
}

}  // namespace perch
