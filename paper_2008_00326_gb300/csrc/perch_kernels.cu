// libperch kernels for sm_103a: observation build (back-projection, CIELAB,
// voxel hash over I), the fused per-hypothesis scorer (fixed-point raster with
// an atomicMin z-buffer in shared memory, resolve with occluder removal and
// image-space down-sampling, warp-cooperative 27-cell radius search,
// CIEDE2000 check, J_r / J_o counts) and the warp-shuffle argmin.
//
// Bit-exactness: every step whose result decides an integer (snapping,
// coverage, depth, back-projection, squared distances, the cylinder test) is
// written with explicit round-to-nearest single-precision intrinsics
// (__fadd_rn, __fmul_rn, __fdiv_rn) and the file is compiled with -fmad=false,
// so no multiply-add is contracted.  Edge functions are exact int32.
#include "perch_internal.cuh"

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

namespace perch {

// ---------------------------------------------------------------------------
// colour: sRGB -> CIELAB (D65) and CIEDE2000 (Sec. IV-B, Eq. 4), binary32
// ---------------------------------------------------------------------------

__device__ float g_srgb_lin[256];   // sRGB decoding of each 8-bit code, filled at start-up

__global__ void k_init_tables()
{
    int i = threadIdx.x;
    if (i < 256) {
        float c = __fdiv_rn((float)i, 255.0f);
        g_srgb_lin[i] = (c <= 0.04045f) ? __fdiv_rn(c, 12.92f)
                                        : powf(__fdiv_rn(__fadd_rn(c, 0.055f), 1.055f), 2.4f);
    }
}

cudaError_t init_device_tables(cudaStream_t s)
{
    k_init_tables<<<1, 256, 0, s>>>();
    return cudaGetLastError();
}

// The colour test only decides whether a difference exceeds tau_c, and the
// parity contract leaves the decisions within 1e-3 of tau_c to rounding (the
// band): the constants' divisions are multiplications by reciprocals, the
// other divisions approximate (__fdividef), the angles in half-turns
// (sinpif / cospif reduce their argument exactly) -- a few 1e-6 relative at
// most, far inside the band.
__device__ __forceinline__ float cie_f(float t)
{
    // cube root above (6/29)^3, the linear toe below it
    return (t > 0.0088564517f) ? cbrtf(t) : (t * 903.29630f + 16.0f) * (1.0f / 116.0f);
}

__device__ __forceinline__ float3 srgb8_to_lab(uint32_t r8, uint32_t g8, uint32_t b8)
{
    float r = g_srgb_lin[r8], g = g_srgb_lin[g8], b = g_srgb_lin[b8];
    float x = 0.4124564f * r + 0.3575761f * g + 0.1804375f * b;
    float y = 0.2126729f * r + 0.7151522f * g + 0.0721750f * b;
    float z = 0.0193339f * r + 0.1191920f * g + 0.9503041f * b;
    float fx = cie_f(x * (1.0f / 0.95047f)), fy = cie_f(y), fz = cie_f(z * (1.0f / 1.08883f));
    return make_float3(116.0f * fy - 16.0f, 500.0f * (fx - fy), 200.0f * (fy - fz));
}

// CIEDE2000 with kL = kC = kH = 1, angles in degrees.
__device__ __forceinline__ float ciede2000(float3 p, float3 q)
{
    const float kDeg = 57.295779513082321f;      // degrees per radian
    const float k25p7 = 6103515625.0f;
    float c1 = sqrtf(p.y * p.y + p.z * p.z);
    float c2 = sqrtf(q.y * q.y + q.z * q.z);
    float cm = 0.5f * (c1 + c2);
    float cm2 = cm * cm, cm7 = cm2 * cm2 * cm2 * cm;
    float g = 0.5f * (1.0f - sqrtf(__fdividef(cm7, cm7 + k25p7)));
    float ap1 = p.y * (1.0f + g), ap2 = q.y * (1.0f + g);
    float cp1 = sqrtf(ap1 * ap1 + p.z * p.z), cp2 = sqrtf(ap2 * ap2 + q.z * q.z);
    float hp1 = (ap1 == 0.0f && p.z == 0.0f) ? 0.0f : atan2f(p.z, ap1) * kDeg;
    float hp2 = (ap2 == 0.0f && q.z == 0.0f) ? 0.0f : atan2f(q.z, ap2) * kDeg;
    if (hp1 < 0.0f) hp1 += 360.0f;
    if (hp2 < 0.0f) hp2 += 360.0f;
    float prod = cp1 * cp2;
    float dh = 0.0f, hm;
    if (prod == 0.0f) {
        hm = hp1 + hp2;
    } else {
        dh = hp2 - hp1;
        if (dh > 180.0f) dh -= 360.0f;
        else if (dh < -180.0f) dh += 360.0f;
        float s = hp1 + hp2;
        if (fabsf(hp1 - hp2) <= 180.0f) hm = 0.5f * s;
        else hm = (s < 360.0f) ? 0.5f * (s + 360.0f) : 0.5f * (s - 360.0f);
    }
    float dL = q.x - p.x;
    float dC = cp2 - cp1;
    float dH = 2.0f * sqrtf(prod) * sinpif(dh * (1.0f / 360.0f));     // sin(dh / 2 degrees)
    float lm = 0.5f * (p.x + q.x) - 50.0f;
    float lm2 = lm * lm;
    float cpm = 0.5f * (cp1 + cp2);
    float t = 1.0f - 0.17f * cospif((hm - 30.0f) * (1.0f / 180.0f)) + 0.24f * cospif(hm * (1.0f / 90.0f))
              + 0.32f * cospif((3.0f * hm + 6.0f) * (1.0f / 180.0f))
              - 0.20f * cospif((4.0f * hm - 63.0f) * (1.0f / 180.0f));
    float e = (hm - 275.0f) * (1.0f / 25.0f);
    float dtheta = 30.0f * __expf(-e * e);
    float cpm2 = cpm * cpm, cpm7 = cpm2 * cpm2 * cpm2 * cpm;
    float rc = 2.0f * sqrtf(__fdividef(cpm7, cpm7 + k25p7));
    float sl = 1.0f + __fdividef(0.015f * lm2, sqrtf(20.0f + lm2));
    float sc = 1.0f + 0.045f * cpm;
    float sh = 1.0f + 0.015f * cpm * t;
    float rt = -sinpif(dtheta * (1.0f / 90.0f)) * rc;                  // sin(2 dtheta degrees)
    float a = __fdividef(dL, sl), b = __fdividef(dC, sc), c = __fdividef(dH, sh);
    return sqrtf(a * a + b * b + c * c + rt * b * c);
}

// ---------------------------------------------------------------------------
// geometry helpers (exact op order)
// ---------------------------------------------------------------------------

// Back-projection of pixel (u,v) at integer depth d (0.1 mm units), Sec. IV-A.
__device__ __forceinline__ float3 back_project(const DevScene& sc, int u, int v, unsigned d)
{
    float z = __fdiv_rn(__uint2float_rn(d), 10000.0f);
    float x = __fdiv_rn(__fmul_rn(__fsub_rn(__int2float_rn(u), sc.cx), z), sc.fx);
    float y = __fdiv_rn(__fmul_rn(__fsub_rn(__int2float_rn(v), sc.cy), z), sc.fy);
    return make_float3(x, y, z);
}

// Hash-cell coordinate floor(x / cell), taken as floor(fl(x * fl(1 / cell))):
// for two points within delta of each other on an axis the two products
// differ by at most delta (1 + 2^-22) / cell + 2 * 1e5 * 2^-24 < 0.997 (cell =
// delta (1 + 1/64), coordinates below 1e5 cells), so their cells are at most
// one apart -- the radius search's 27 cells hold every point within delta.
__device__ __forceinline__ int cell_coord(float x, float inv_cell)
{
    return __float2int_rd(__fmul_rn(x, inv_cell));
}

__device__ __forceinline__ unsigned long long cell_key(int cx, int cy, int cz)
{
    return ((unsigned long long)((unsigned)(cx + kCellBias) & 0x1FFFFFu) << 42) |
           ((unsigned long long)((unsigned)(cy + kCellBias) & 0x1FFFFFu) << 21) |
           (unsigned long long)((unsigned)(cz + kCellBias) & 0x1FFFFFu);
}

__device__ __forceinline__ uint32_t hash_slot(unsigned long long k, uint32_t mask)
{
    k ^= k >> 31;
    k *= 0x7fb5d329728ea185ull;
    k ^= k >> 27;
    k *= 0x81dadef4bc2dd44dull;
    k ^= k >> 33;
    return (uint32_t)k & mask;
}

// ---------------------------------------------------------------------------
// observation build: per-pixel CIELAB, cloud I, voxel hash (cell = delta*(1+1/64))
// ---------------------------------------------------------------------------

__global__ void k_obs_insert(DevScene sc, const uint8_t* __restrict__ rgb, float4* lab, float4* pxyz,
                             int32_t* slot_of_pixel, unsigned long long* keys, uint32_t* count,
                             uint32_t mask, int* n_valid, int* err)
{
    int npx = sc.W * sc.H;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npx) return;
    int u = i % sc.W, v = i / sc.W;
    float3 L = srgb8_to_lab(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2]);
    lab[i] = make_float4(L.x, L.y, L.z, 0.0f);
    unsigned d = sc.depth[i];
    int slot = -1;
    pxyz[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (d != 0 && u % sc.stride == 0 && v % sc.stride == 0) {
        float3 p = back_project(sc, u, v, d);
        pxyz[i] = make_float4(p.x, p.y, p.z, 1.0f);
        unsigned long long k = cell_key(cell_coord(p.x, sc.inv_cell), cell_coord(p.y, sc.inv_cell),
                                        cell_coord(p.z, sc.inv_cell));
        uint32_t h = hash_slot(k, mask);
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            unsigned long long prev = atomicCAS(&keys[h], kEmptyKey, k);
            if (prev == kEmptyKey || prev == k) {
                slot = (int)h;
                break;
            }
            h = (h + 1) & mask;
        }
        if (slot < 0) atomicOr(err, kErrHashFull);
        else atomicAdd(&count[slot], 1u);
        atomicAdd(n_valid, 1);
    }
    slot_of_pixel[i] = slot;
}

// Exclusive scan of count[0..n) into start[], in tiles of 1024 (one block per
// tile), then a second pass over the tile sums, then the offsets.
__device__ __forceinline__ uint32_t block_incl_scan_1024(uint32_t x, uint32_t* warp_sums)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    if (w > 0) x += warp_sums[w - 1];
    return x;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t* count, uint32_t* start,
                                                    uint32_t* tile_sums, uint32_t n)
{
    __shared__ uint32_t ws[32];
    uint32_t i = blockIdx.x * 1024u + threadIdx.x;
    uint32_t x = i < n ? count[i] : 0u;
    uint32_t incl = block_incl_scan_1024(x, ws);
    if (i < n) start[i] = incl - x;
    if (threadIdx.x == 1023) tile_sums[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(1024) k_scan_sums(uint32_t* tile_sums, uint32_t n_tiles)
{
    // n_tiles <= 1024 * k; sequential over chunks of 1024
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n_tiles; base += 1024) {
        uint32_t i = base + threadIdx.x;
        uint32_t x = i < n_tiles ? tile_sums[i] : 0u;
        uint32_t incl = block_incl_scan_1024(x, ws);
        uint32_t c = carry;
        if (i < n_tiles) tile_sums[i] = c + incl - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + incl;
        __syncthreads();
    }
}

__global__ void k_finish_table(const unsigned long long* keys, const uint32_t* count,
                               uint32_t* start, const uint32_t* tile_offsets, uint4* table,
                               uint32_t n)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t s = start[i] + tile_offsets[i >> 10];
    start[i] = s;
    unsigned long long k = keys[i];
    table[i] = make_uint4((uint32_t)k, (uint32_t)(k >> 32), s, k == kEmptyKey ? 0u : count[i]);
}

// Re-insert the occupied slots of the build table into a table sized for
// them (twice the occupied count, rounded up to a power of two), so that the
// lookups of the radius search touch a compact, cache-friendly array.
__global__ void k_compact_table(const uint4* big, uint32_t cap_big, uint4* small, uint32_t mask,
                                int* err)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap_big) return;
    uint4 e = big[i];
    unsigned long long k = (unsigned long long)e.x | ((unsigned long long)e.y << 32);
    if (k == kEmptyKey) return;
    uint32_t h = hash_slot(k, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(&small[h]), kEmptyKey, k);
        if (prev == kEmptyKey) {
            small[h].z = e.z;
            small[h].w = e.w;
            return;
        }
        h = (h + 1) & mask;
    }
    atomicOr(err, kErrHashFull);
}

// ---- near-cell bitmap: lets a query whose 27 neighbour cells are all empty
// skip the hash lookups (exact: such a query has no candidate at all)

__global__ void k_cell_bounds(DevScene sc, int* bounds)
{
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sc.n_pts; i += gridDim.x * blockDim.x) {
        const float4 p = sc.pts[i];
        const int c[3] = {cell_coord(p.x, sc.inv_cell), cell_coord(p.y, sc.inv_cell), cell_coord(p.z, sc.inv_cell)};
#pragma unroll
        for (int a = 0; a < 3; ++a) { lo[a] = min(lo[a], c[a]); hi[a] = max(hi[a], c[a]); }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) { atomicMin(&bounds[a], lo[a]); atomicMax(&bounds[3 + a], hi[a]); }
    }
}

__device__ __forceinline__ long long near_index(const DevScene& sc, int x, int y, int z)
{
    const int ix = x - sc.near_lo[0], iy = y - sc.near_lo[1], iz = z - sc.near_lo[2];
    if (ix < 0 || iy < 0 || iz < 0 || ix >= sc.near_n[0] || iy >= sc.near_n[1] || iz >= sc.near_n[2]) return -1;
    return ((long long)iz * sc.near_n[1] + iy) * sc.near_n[0] + ix;
}

__global__ void k_cell_occupancy(DevScene sc, uint32_t* occ)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sc.n_pts; i += gridDim.x * blockDim.x) {
        const float4 p = sc.pts[i];
        const long long b = near_index(sc, cell_coord(p.x, sc.inv_cell), cell_coord(p.y, sc.inv_cell),
                                       cell_coord(p.z, sc.inv_cell));
        if (b >= 0) atomicOr(&occ[b >> 5], 1u << (b & 31));
    }
}

__global__ void k_cell_dilate(DevScene sc, const uint32_t* occ, uint32_t* near_bits)
{
    const long long n = (long long)sc.near_n[0] * sc.near_n[1] * sc.near_n[2];
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < n;
         b += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(b % sc.near_n[0]) + sc.near_lo[0];
        const int y = (int)((b / sc.near_n[0]) % sc.near_n[1]) + sc.near_lo[1];
        const int z = (int)(b / ((long long)sc.near_n[0] * sc.near_n[1])) + sc.near_lo[2];
        bool any = false;
        for (int k = 0; k < 27 && !any; ++k) {
            const long long q = near_index(sc, x + k % 3 - 1, y + (k / 3) % 3 - 1, z + k / 9 - 1);
            any = q >= 0 && ((occ[q >> 5] >> (q & 31)) & 1u);
        }
        if (any) atomicOr(&near_bits[b >> 5], 1u << (b & 31));
    }
}

cudaError_t launch_cell_bounds(const DevScene& sc, int* bounds, cudaStream_t s)
{
    if (sc.n_pts <= 0) return cudaSuccess;
    k_cell_bounds<<<min(1024, (sc.n_pts + 255) / 256), 256, 0, s>>>(sc, bounds);
    return cudaGetLastError();
}

cudaError_t launch_near_cells(const DevScene& sc, uint32_t* occ, uint32_t* near_bits, cudaStream_t s)
{
    if (sc.n_pts <= 0) return cudaSuccess;
    k_cell_occupancy<<<min(1024, (sc.n_pts + 255) / 256), 256, 0, s>>>(sc, occ);
    const long long n = (long long)sc.near_n[0] * sc.near_n[1] * sc.near_n[2];
    k_cell_dilate<<<(unsigned)std::min<long long>(4096, (n + 255) / 256), 256, 0, s>>>(sc, occ, near_bits);
    return cudaGetLastError();
}

// ---- dense cell index: count per cell, exclusive scan, scatter by cell

__global__ void k_dense_count(DevScene sc, uint32_t* count)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sc.n_pts; i += gridDim.x * blockDim.x) {
        const float4 p = sc.pts[i];
        const long long c = near_index(sc, cell_coord(p.x, sc.inv_cell), cell_coord(p.y, sc.inv_cell),
                                       cell_coord(p.z, sc.inv_cell));
        if (c >= 0) atomicAdd(&count[c], 1u);
    }
}

__global__ void k_add_tile_offsets(uint32_t* start, const uint32_t* tile_offsets, uint32_t n)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) start[i] += tile_offsets[i >> 10];
}

__global__ void k_dense_scatter(DevScene sc, const uint32_t* start, uint32_t* cursor, float4* out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sc.n_pts; i += gridDim.x * blockDim.x) {
        const float4 p = sc.pts[i];
        const long long c = near_index(sc, cell_coord(p.x, sc.inv_cell), cell_coord(p.y, sc.inv_cell),
                                       cell_coord(p.z, sc.inv_cell));
        if (c >= 0) out[start[c] + atomicAdd(&cursor[c], 1u)] = p;
    }
}

cudaError_t launch_dense_cells(const DevScene& sc, uint32_t* count, uint32_t* cursor, uint32_t* tile_sums,
                               uint32_t* cell_start, float4* out, cudaStream_t s)
{
    const long long n = (long long)sc.near_n[0] * sc.near_n[1] * sc.near_n[2];
    if (sc.n_pts <= 0 || n <= 0 || n > 0xFFFFFFFFll) return cudaErrorInvalidValue;
    const unsigned blocks_pts = (unsigned)std::min(1024, (sc.n_pts + 255) / 256);
    k_dense_count<<<blocks_pts, 256, 0, s>>>(sc, count);
    const uint32_t n_tiles = (uint32_t)((n + 1023) / 1024);
    k_scan_tiles<<<n_tiles, 1024, 0, s>>>(count, cell_start, tile_sums, (uint32_t)n);
    k_scan_sums<<<1, 1024, 0, s>>>(tile_sums, n_tiles);
    k_add_tile_offsets<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cell_start, tile_sums, (uint32_t)n);
    k_dense_scatter<<<blocks_pts, 256, 0, s>>>(sc, cell_start, cursor, out);
    return cudaGetLastError();
}

cudaError_t launch_compact_table(const uint4* big, uint32_t cap_big, uint4* small, uint32_t cap_small,
                                 int* err, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(small, 0xFF, sizeof(uint4) * cap_small, s);
    if (e != cudaSuccess) return e;
    k_compact_table<<<(cap_big + 255) / 256, 256, 0, s>>>(big, cap_big, small, cap_small - 1, err);
    return cudaGetLastError();
}

__global__ void k_count_cells(const uint4* table, uint32_t n, int* n_cells)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    bool occ = false;
    if (i < n) {
        uint4 e = table[i];
        occ = !(e.x == 0xFFFFFFFFu && e.y == 0xFFFFFFFFu);
    }
    unsigned b = __ballot_sync(0xffffffffu, occ);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_cells, __popc(b));
}

__global__ void k_obs_scatter(DevScene sc, const int32_t* slot_of_pixel, const uint32_t* start,
                              uint32_t* cursor, float4* pts)
{
    int npx = sc.W * sc.H;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npx) return;
    int slot = slot_of_pixel[i];
    if (slot < 0) return;
    int u = i % sc.W, v = i / sc.W;
    float3 p = back_project(sc, u, v, sc.depth[i]);
    uint32_t pos = start[slot] + atomicAdd(&cursor[slot], 1u);
    // the pixel as (v << 16 | u): ordered like the index v W + u, and its
    // coordinates come back without a division
    pts[pos] = make_float4(p.x, p.y, p.z, __uint_as_float(((uint32_t)v << 16) | (uint32_t)u));
}

cudaError_t launch_build(const DevScene& sc, const BuildBuffers& b, uint32_t cap,
                         const uint8_t* rgb_dev, int* err, cudaStream_t s)
{
    int npx = sc.W * sc.H;
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.keys, 0xFF, sizeof(unsigned long long) * cap, s))) return e;
    if ((e = cudaMemsetAsync(b.count, 0, sizeof(uint32_t) * cap, s))) return e;
    if ((e = cudaMemsetAsync(b.cursor, 0, sizeof(uint32_t) * cap, s))) return e;
    if ((e = cudaMemsetAsync(b.n_valid, 0, 2 * sizeof(int), s))) return e;
    int blocks = (npx + 255) / 256;
    k_obs_insert<<<blocks, 256, 0, s>>>(sc, rgb_dev, b.lab, b.pxyz, b.slot_of_pixel, b.keys, b.count,
                                        cap - 1, b.n_valid, err);
    uint32_t n_tiles = (cap + 1023) / 1024;
    // the tile sums of the scan live just past the cursors
    uint32_t* tile_sums = b.cursor + cap;   // BuildBuffers::cursor has cap + n_tiles words
    k_scan_tiles<<<n_tiles, 1024, 0, s>>>(b.count, b.start, tile_sums, cap);
    k_scan_sums<<<1, 1024, 0, s>>>(tile_sums, n_tiles);
    k_finish_table<<<(cap + 255) / 256, 256, 0, s>>>(b.keys, b.count, b.start, tile_sums, b.table,
                                                     cap);
    k_obs_scatter<<<blocks, 256, 0, s>>>(sc, b.slot_of_pixel, b.start, b.cursor, b.pts);
    k_count_cells<<<(cap + 255) / 256, 256, 0, s>>>(b.table, cap, b.n_valid + 1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// scoring kernel
// ---------------------------------------------------------------------------


struct TriSetup {
    int x[3], y[3];               // snapped positions, 1/16 px
    float iz[3];                  // 1/Z
    int vid[3];                   // mesh vertex ids after the orientation swap
    int A;                        // doubled area > 0
};

struct __align__(16) TriStage {   // a set-up triangle staged for its warp (64 bytes, 4 x 16-byte moves)
    // edge i at the sample of pixel (u, v): a[i] u + b[i] v + c[i] + bias_i
    // (two's-complement arithmetic, exact), bias_i = 1 unless edge i owns
    // the samples lying on it; covered iff every a[i] u + b[i] v + c[i] >= 0
    int a[3], b[3], c[3];
    float iz[3];                  // 1/Z
    int A, tri;                   // doubled area, triangle id
    int uv0;                      // pixel box origin u0 | v0 << 16
    int bw_bias;                  // box width | bias bits << 16
};

__device__ __forceinline__ int edge_fn(int ax, int ay, int bx, int by, int px, int py)
{
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

__device__ __forceinline__ bool owns(int dx, int dy)
{
    return dy > 0 || (dy == 0 && dx < 0);
}

__device__ __forceinline__ int floor16(int x) { return x >> 4; }         // arithmetic shift
__device__ __forceinline__ int ceil16(int x) { return -((-x) >> 4); }

// Bit i set iff edge i of the oriented triangle (edge 0: vertex 1 -> 2, edge
// 1: 2 -> 0, edge 2: 0 -> 1) owns the samples lying on it.
__device__ __forceinline__ int owns_of(const TriSetup& o)
{
    return (owns(o.x[2] - o.x[1], o.y[2] - o.y[1]) ? 1 : 0) | (owns(o.x[0] - o.x[2], o.y[0] - o.y[2]) ? 2 : 0) |
           (owns(o.x[1] - o.x[0], o.y[1] - o.y[0]) ? 4 : 0);
}

// Doubled area and orientation of a loaded triangle: a negative area swaps
// vertices 1 and 2 (two-sided rendering).  False if degenerate (A == 0).
__device__ __forceinline__ bool orient_triangle(TriSetup& o)
{
    int A = edge_fn(o.x[0], o.y[0], o.x[1], o.y[1], o.x[2], o.y[2]);
    if (A == 0) return false;
    if (A < 0) {
        int tx = o.x[1], ty = o.y[1], tvid = o.vid[1];
        float ti = o.iz[1];
        o.x[1] = o.x[2]; o.y[1] = o.y[2]; o.iz[1] = o.iz[2]; o.vid[1] = o.vid[2];
        o.x[2] = tx; o.y[2] = ty; o.iz[2] = ti; o.vid[2] = tvid;
        A = -A;
    }
    o.A = A;
    return true;
}

// Triangle loaded at a pose: transform, near/guard-band cull, projection,
// 4-bit snap (orient_triangle completes the set-up).  False if culled.
__device__ __forceinline__ bool load_triangle(const DevScene& sc, const DevMesh& m,
                                              const float* P, int4 tv, TriSetup& o)
{
    int vids[3] = {tv.x, tv.y, tv.z};
    const float gx0 = (float)(-16 * sc.W), gx1 = (float)(32 * sc.W);
    const float gy0 = (float)(-16 * sc.H), gy1 = (float)(32 * sc.H);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float4 v = __ldg(&m.verts[vids[k]]);
        float X = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P[0], v.x), __fmul_rn(P[1], v.y)),
                                      __fmul_rn(P[2], v.z)), P[3]);
        float Y = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P[4], v.x), __fmul_rn(P[5], v.y)),
                                      __fmul_rn(P[6], v.z)), P[7]);
        float Z = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P[8], v.x), __fmul_rn(P[9], v.y)),
                                      __fmul_rn(P[10], v.z)), P[11]);
        if (!(Z >= sc.z_near)) return false;
        float px = __fadd_rn(__fmul_rn(sc.fx, __fdiv_rn(X, Z)), sc.cx);
        float py = __fadd_rn(__fmul_rn(sc.fy, __fdiv_rn(Y, Z)), sc.cy);
        float sx = __fmul_rn(px, 16.0f), sy = __fmul_rn(py, 16.0f);
        if (!(sx >= gx0) || !(sx < gx1) || !(sy >= gy0) || !(sy < gy1)) return false;
        o.x[k] = __float2int_rn(sx);
        o.y[k] = __float2int_rn(sy);
        o.iz[k] = __frcp_rn(Z);        // = fl(1 / Z), as the division would give
        o.vid[k] = vids[k];
    }
    return true;
}

// Depth of a covered sample from the edge values (perspective-correct:
// z = A / (w0/Z0 + w1/Z1 + w2/Z2), one division).
// Returns false if the depth falls outside [1, 2^32-1].
__device__ __forceinline__ bool sample_depth(int w0, int w1, int w2, const float* iz, int A,
                                             unsigned& d)
{
    float num = __fadd_rn(__fadd_rn(__fmul_rn(__int2float_rn(w0), iz[0]),
                                    __fmul_rn(__int2float_rn(w1), iz[1])),
                          __fmul_rn(__int2float_rn(w2), iz[2]));
    float z = __fdiv_rn(__int2float_rn(A), num);
    float dz = __fmul_rn(z, 10000.0f);
    // z >= 0 here (A > 0 and every 1/Z > 0), so dz in [0, 2^32) rounds to
    // nearest in 32 bits (the largest binary32 below 2^32 is an integer)
    if (!(dz < 4294967296.0f)) return false;
    d = __float2uint_rn(dz);
    return d >= 1u;
}

template <bool K32>
__device__ __forceinline__ void zmin(uint32_t* zbuf, int idx, unsigned d, int tri, int* err)
{
    if (K32) {
        if (d > 0xFFFFu) {
            atomicOr(err, kErrKeyRange);
            return;
        }
        atomicMin(&zbuf[idx], (d << 16) | (unsigned)tri);
    } else {
        unsigned long long* z64 = reinterpret_cast<unsigned long long*>(zbuf);
        atomicMin(&z64[idx], ((unsigned long long)d << 32) | (unsigned)tri);
    }
}

// ---- resolve queue and per-warp cell groups -------------------------------

constexpr int kWarpQueue = 64;    // kept rendered points queued per warp (a ring)
constexpr int kGroups = 1;        // distinct query cells looked up together per warp

// A group of G queries shares a 27-cell candidate list; k = floor(32 / G)
// lanes test each query's candidates.  Lane l serves query floor(l / k),
// taken as (l * ceil(1024 / k)) >> 10 (exact for l < 32 and k <= 32), so the
// split needs no integer division.
__constant__ unsigned char c_lanes_per_query[33] = {
    32, 32, 16, 10, 8, 6, 5, 4, 4, 3, 3, 2, 2, 2, 2, 2, 2,
    1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
__constant__ unsigned short c_lane_div[33] = {
    1024, 1024, 512, 342, 256, 205, 171, 147, 128, 114, 103, 94, 86, 79, 74, 69, 64,
    61, 57, 54, 52, 49, 47, 45, 43, 41, 40, 38, 37, 36, 35, 34, 32};

struct __align__(16) KeptPoint {  // a rendered point of R \ C waiting for its radius search
    float x, y, z;
    uint32_t pix;                 // its pixel u | v << 16 (the colour is interpolated only if needed)
};

// Per-warp scratch of the radius search (shared memory).
struct __align__(16) WarpProbe {
    int2 runs[kGroups][27];       // per group: non-empty runs as (start - first pair index, end pair index)
    int total[kGroups];           // per group: candidates in its 27 cells
    unsigned mask[kGroups];       // per group: lanes whose query lies in the group's cell
    unsigned char qlist[kGroups][32];  // per group: the lanes of its queries, in lane order
    float4 q[32];                 // query of each lane
    unsigned long long best[32];  // nearest-neighbour key of each lane's query
    float4 stage[64];             // a chunk of the group's candidates, shared by its queries
};

// Per-warp scratch: the radius search and the rasteriser's triangle stage
// use the same bytes (the two phases are separated by block barriers).
constexpr size_t kWarpScratch = sizeof(WarpProbe) > 32 * sizeof(TriStage) ? sizeof(WarpProbe)
                                                                            : 32 * sizeof(TriStage);
static_assert(sizeof(KeptPoint) == 16, "kept-point queue entries are 16 bytes");
static_assert(sizeof(TriStage) == 64, "staged triangles are 64 bytes");
static_assert(kWarpScratch % 16 == 0, "per-warp scratch keeps 16-byte alignment");
static_assert(sizeof(WarpProbe) % 16 == 0, "per-warp scratch keeps 16-byte alignment");

// Warp-cooperative lookup of the 27-cell neighbourhoods of up to kGroups
// query cells at once.  With the dense cell index, lane j < 9 reads the two
// bounds of one row's three cells (they are contiguous); otherwise lane
// j < 27 probes the hash table for neighbour j, issuing all first-slot loads
// before resolving any (the table lives in L2, so the loads overlap).  Group
// g's non-empty runs are stored in order with a running candidate count so
// that candidate i of the group is point runs[r].x + i for the first run r
// with i < runs[r].y.
__device__ __forceinline__ void lookup_cells(const DevScene& sc, const int* gx, const int* gy,
                                             const int* gz, int ng, WarpProbe& W, int lane, int* nruns)
{
    const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
        if (g >= ng) break;
        uint32_t start = 0, cnt = 0;
        if (sc.cell_start) {
            // dense index: lane j < 9 takes row (y + j % 3 - 1, z + j / 3 - 1),
            // whose cells x-1..x+1 are one run of the cell-sorted points
            if (lane < 9) {
                const int ry = gy[g] + lane % 3 - 1 - sc.near_lo[1], rz = gz[g] + lane / 3 - 1 - sc.near_lo[2];
                const int x0 = max(gx[g] - 1 - sc.near_lo[0], 0), x1 = min(gx[g] + 1 - sc.near_lo[0], sc.near_n[0] - 1);
                if (ry >= 0 && ry < sc.near_n[1] && rz >= 0 && rz < sc.near_n[2] && x0 <= x1) {
                    const long long row = ((long long)rz * sc.near_n[1] + ry) * sc.near_n[0];
                    start = __ldg(&sc.cell_start[row + x0]);
                    cnt = __ldg(&sc.cell_start[row + x1 + 1]) - start;
                }
            }
        } else if (lane < 27) {
            // voxel hash (a cell box too large for the dense index): lane j
            // probes the table for neighbour j
            const unsigned long long key = cell_key(gx[g] + dx, gy[g] + dy, gz[g] + dz);
            uint32_t slot = hash_slot(key, sc.table_mask);
            for (uint32_t probe = 0; probe <= sc.table_mask; ++probe) {
                const uint4 x = __ldg(&sc.table[slot]);
                unsigned long long k = (unsigned long long)x.x | ((unsigned long long)x.y << 32);
                if (k == key) {
                    start = x.z;
                    cnt = x.w;
                    break;
                }
                if (k == kEmptyKey) break;
                slot = (slot + 1) & sc.table_mask;
            }
        }
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const unsigned nonempty = __ballot_sync(0xffffffffu, cnt != 0);
        if (cnt != 0)
            W.runs[g][__popc(nonempty & ((1u << lane) - 1u))] =
                make_int2((int)start - (int)(incl - cnt), (int)incl);
        if (lane == 31) W.total[g] = (int)incl;
        nruns[g] = __popc(nonempty);
    }
}

// Radius search for up to 32 queued points (one per lane; `valid` marks the
// lanes holding one).  Lanes whose points fall in the same hash cell form a
// group (__match_any_sync); each group's 27-cell neighbourhood is looked up
// once, cooperatively.  The group's candidates are then staged in shared
// memory 64 at a time (two coalesced loads per lane, each candidate loaded
// once however many of the group's queries test it) and tested by all 32
// lanes: floor(32 / G) lanes per query (G = the group's queries) split each
// chunk, each keeps its minimum (d2 bits, pixel) in a register and folds it
// into the query's result with one shared-memory atomicMin.  Returns the
// lane's own result: the nearest observed point within delta (smallest FP32
// squared distance, ties to the lowest pixel index) or kEmptyKey.  All 32
// lanes must call it.
// Admissible band of the observed-side keys (jo_mode 1: for every observed
// point of the band, the key (d2 bits << 32 | rendered pixel) of its nearest
// rendered point within delta, kEmptyKey if none).
struct MarkBand {
    uint32_t* marks;
    int u0, u1, v0, v1, vw;
    int* err;                     // debug builds: where index violations are reported
};

// Candidates j, j + k, ... of a staged chunk of n against query q, folded
// into local: the minimum (d2 bits << 32 | pixel) within delta, or kEmptyKey.
// MARK (jo_mode 1) also folds the pair into the key of every observed point
// within delta that lies in the admissible band: its nearest rendered point
// is the smallest (d2, rendered pixel), the rendered pixel carried in q.w.
template <bool MARK>
__device__ __forceinline__ unsigned long long scan_staged(const DevScene& sc, const float4 q, const float4* stage,
                                                          int n, int j, int k, const MarkBand& mb,
                                                          unsigned long long local)
{
    for (int i = j; i < n; i += k) {
        const float4 c = stage[i];
        float ex = __fsub_rn(q.x, c.x), ey = __fsub_rn(q.y, c.y), ez = __fsub_rn(q.z, c.z);
        float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
        if (d2 <= sc.delta2) {
            unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | __float_as_uint(c.w);
            local = key < local ? key : local;
            if (MARK) {
                const uint32_t pw = __float_as_uint(c.w);
                const int pu = (int)(pw & 0xFFFFu), pv = (int)(pw >> 16);
                if (pu >= mb.u0 && pu < mb.u1 && pv >= mb.v0 && pv < mb.v1) {
                    const int i = (pv - mb.v0) * mb.vw + (pu - mb.u0);
                    atomicMin(reinterpret_cast<unsigned long long*>(mb.marks) + i,
                              ((unsigned long long)__float_as_uint(d2) << 32) | __float_as_uint(q.w));
                }
            }
        }
    }
    return local;
}

// Candidates c0 .. c0 + 63 of a group's runs staged in the warp's shared
// memory (two coalesced loads per lane).  Lane j < (the group's run count)
// holds run j as run = (start - first candidate index, end candidate index)
// (the other lanes: end = INT_MAX); the run of candidate c is the first whose
// end exceeds c, found by a five-step binary search over the lanes.
__device__ __forceinline__ int candidate_point(int2 run, int c)
{
    int r = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int e = __shfl_sync(0xffffffffu, run.y, r + step - 1);
        if (e <= c) r += step;
    }
    return __shfl_sync(0xffffffffu, run.x, r) + c;
}

__device__ __forceinline__ void stage_chunk(const DevScene& sc, WarpProbe& W, int2 run, int c0, int T, int lane,
                                            int* err)
{
    const int ci = c0 + lane, cj = ci + 32;
    const int pi = candidate_point(run, ci), pj = candidate_point(run, cj);
    if (ci < T && PERCH_CHECKED((unsigned)pi < (unsigned)sc.n_pts, err)) W.stage[lane] = __ldg(&sc.pts[pi]);
    if (cj < T && PERCH_CHECKED((unsigned)pj < (unsigned)sc.n_pts, err)) W.stage[lane + 32] = __ldg(&sc.pts[pj]);
}

template <bool MARK>
__device__ unsigned long long probe_batch(const DevScene& sc, bool valid, float qx, float qy,
                                          float qz, uint32_t qpix, WarpProbe& W, int lane, const MarkBand& mb)
{
    int cx = 0, cy = 0, cz = 0;
    unsigned long long key = kEmptyKey;
    if (valid) {
        cx = cell_coord(qx, sc.inv_cell);
        cy = cell_coord(qy, sc.inv_cell);
        cz = cell_coord(qz, sc.inv_cell);
        if (sc.near_bits) {
            // no observed point in the 27 cells: nothing to look up
            const long long b = near_index(sc, cx, cy, cz);
            valid = b >= 0 && ((__ldg(&sc.near_bits[b >> 5]) >> (b & 31)) & 1u);
        }
        if (valid) key = cell_key(cx, cy, cz);
    }
    W.q[lane] = make_float4(qx, qy, qz, __uint_as_float(qpix));
    W.best[lane] = kEmptyKey;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(grp) - 1;
    const unsigned leaders = __ballot_sync(0xffffffffu, valid && lane == leader);
    const int my_g = __popc(leaders & ((1u << leader) - 1u));
    const int my_pos = __popc(grp & ((1u << lane) - 1u));
    unsigned rest = leaders;
    for (int g0 = 0; rest != 0; g0 += kGroups) {
        int gx[kGroups], gy[kGroups], gz[kGroups];
        int ng = 0;
#pragma unroll
        for (int g = 0; g < kGroups; ++g) {
            gx[g] = gy[g] = gz[g] = 0;
            if (rest != 0) {
                const int L = __ffs(rest) - 1;
                rest &= rest - 1;
                gx[g] = __shfl_sync(0xffffffffu, cx, L);
                gy[g] = __shfl_sync(0xffffffffu, cy, L);
                gz[g] = __shfl_sync(0xffffffffu, cz, L);
                const unsigned m = __shfl_sync(0xffffffffu, grp, L);
                if (lane == 0) W.mask[g] = m;
                ng = g + 1;
            }
        }
        if (valid && my_g >= g0 && my_g < g0 + kGroups) W.qlist[my_g - g0][my_pos] = (unsigned char)lane;
        int nruns[kGroups];
        lookup_cells(sc, gx, gy, gz, ng, W, lane, nruns);
        __syncwarp();
        for (int g = 0; g < ng; ++g) {
            const int T = W.total[g];
            if (T == 0) continue;
            // k = floor(32 / G) lanes per query; lane j of a query takes
            // candidates j, j + k, ... of each staged chunk and keeps its
            // minimum in a register
            const int G = __popc(W.mask[g]);
            const int k = c_lanes_per_query[G];
            const int qj = (lane * (int)c_lane_div[k]) >> 10;
            const bool active = lane < G * k;
            const int ql = active ? W.qlist[g][qj] : 0;
            const float4 q = W.q[ql];
            unsigned long long local = kEmptyKey;
            const int2 run = lane < nruns[g] ? W.runs[g][lane] : make_int2(0, INT_MAX);
            for (int c0 = 0; c0 < T; c0 += 64) {
                stage_chunk(sc, W, run, c0, T, lane, mb.err);
                __syncwarp();
                const int n = min(64, T - c0);
                if (active)
                    local = scan_staged<MARK>(sc, q, W.stage, n, lane - qj * k, k, mb, local);
                __syncwarp();
            }
            if (active && local != kEmptyKey) atomicMin(&W.best[ql], local);
        }
        __syncwarp();
    }
    return W.best[lane];
}

// Conservative pixel box of an object-frame box [lo,hi] at pose P (2 px
// margin), clipped to [cu0,cu1) x [cv0,cv1).  Falls back to the clip box
// when a corner is not in front of the camera.  Also returns the largest Z.
__device__ void project_box(const DevScene& sc, const float* P, const float* lo, const float* hi,
                            int cu0, int cv0, int cu1, int cv1, int* box, float* zmax)
{
    float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f, zm = -3.0e38f;
    bool ok = true;
    for (int c = 0; c < 8; ++c) {
        float x = (c & 1) ? hi[0] : lo[0];
        float y = (c & 2) ? hi[1] : lo[1];
        float z = (c & 4) ? hi[2] : lo[2];
        float X = P[0] * x + P[1] * y + P[2] * z + P[3];
        float Y = P[4] * x + P[5] * y + P[6] * z + P[7];
        float Z = P[8] * x + P[9] * y + P[10] * z + P[11];
        zm = fmaxf(zm, Z);
        if (!(Z > 1e-4f)) {
            ok = false;
            continue;
        }
        float u = sc.fx * (X / Z) + sc.cx, v = sc.fy * (Y / Z) + sc.cy;
        umin = fminf(umin, u); umax = fmaxf(umax, u);
        vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
    }
    *zmax = zm;
    if (!ok || !(umax - umin < 1.0e7f) || !(vmax - vmin < 1.0e7f)) {
        box[0] = cu0; box[1] = cv0; box[2] = cu1; box[3] = cv1;
        return;
    }
    int u0 = (int)floorf(fmaxf(umin, -1.0e7f)) - 2, u1 = (int)ceilf(fminf(umax, 1.0e7f)) + 3;
    int v0 = (int)floorf(fmaxf(vmin, -1.0e7f)) - 2, v1 = (int)ceilf(fminf(vmax, 1.0e7f)) + 3;
    box[0] = max(u0, cu0); box[1] = max(v0, cv0);
    box[2] = min(u1, cu1); box[3] = min(v1, cv1);
    if (box[2] < box[0]) box[2] = box[0];
    if (box[3] < box[1]) box[3] = box[1];
}

// Shared-memory carve-up of one scoring block.
struct ScoreSmem {
    uint32_t* zbuf;               // z-buffer tile (32- or 64-bit keys)
    uint32_t* marks;              // admissible-band bitset
    KeptPoint* kept;              // per warp: resolve -> radius-search ring queue
    WarpProbe* probe;             // per warp scratch of the radius search (aliases stage)
    TriStage* stage;              // per warp 32 staged triangles (aliases probe)
    int* next_batch;
    int* refused;                 // tree edges: the object would occlude a placed one
    int* bin_cnt;                 // kBinTiles: triangles binned per z-buffer tile
    int* jo_next;                 // plain scoring: next chunk of J_o's |I cap V|
    int* raster_done;             // plain scoring: warps done with the tile's raster
    int* vbounds;                 // snapped vertex bounds of the hypothesis (vertex_pass)
};

// ---- per-hypothesis vertex cache (one slot of global scratch per block) ----
//
// Each vertex is transformed, projected and snapped once per hypothesis and
// kept as (x16 : int16, y16 : int16, 1/Z : float); a vertex that fails the
// near-plane or guard-band test is stored with x16 = -32768, which culls every
// triangle that uses it.  Used when 32 W and 32 H fit in int16.
constexpr int kCulledX = -32768;

//
// bounds (optional, shared memory, initialised to INT_MAX, INT_MAX, INT_MIN,
// INT_MIN): the smallest and largest snapped x and y of the vertices kept.
__device__ __forceinline__ void vertex_pass(const DevScene& sc, const DevMesh& m, const float* P,
                                            unsigned long long* vc, int nt, int* bounds = nullptr)
{
    const float gx0 = (float)(-16 * sc.W), gx1 = (float)(32 * sc.W);
    const float gy0 = (float)(-16 * sc.H), gy1 = (float)(32 * sc.H);
    int xmin = INT_MAX, ymin = INT_MAX, xmax = INT_MIN, ymax = INT_MIN;
#pragma unroll 2
    for (int i = threadIdx.x; i < m.n_verts; i += nt) {
        float4 v = __ldg(&m.verts[i]);
        float X = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P[0], v.x), __fmul_rn(P[1], v.y)),
                                      __fmul_rn(P[2], v.z)), P[3]);
        float Y = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P[4], v.x), __fmul_rn(P[5], v.y)),
                                      __fmul_rn(P[6], v.z)), P[7]);
        float Z = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P[8], v.x), __fmul_rn(P[9], v.y)),
                                      __fmul_rn(P[10], v.z)), P[11]);
        unsigned long long rec = (unsigned long long)(uint16_t)kCulledX;
        if (Z >= sc.z_near) {
            float sx = __fmul_rn(__fadd_rn(__fmul_rn(sc.fx, __fdiv_rn(X, Z)), sc.cx), 16.0f);
            float sy = __fmul_rn(__fadd_rn(__fmul_rn(sc.fy, __fdiv_rn(Y, Z)), sc.cy), 16.0f);
            if (sx >= gx0 && sx < gx1 && sy >= gy0 && sy < gy1) {
                const int xi = __float2int_rn(sx), yi = __float2int_rn(sy);
                xmin = min(xmin, xi); xmax = max(xmax, xi);
                ymin = min(ymin, yi); ymax = max(ymax, yi);
                uint32_t xs = (uint16_t)(int16_t)xi;
                uint32_t ys = (uint16_t)(int16_t)yi;
                rec = (unsigned long long)(xs | (ys << 16)) |
                      ((unsigned long long)__float_as_uint(__frcp_rn(Z)) << 32);
            }
        }
        vc[i] = rec;
    }
    if (bounds) {
        xmin = __reduce_min_sync(0xffffffffu, xmin);
        ymin = __reduce_min_sync(0xffffffffu, ymin);
        xmax = __reduce_max_sync(0xffffffffu, xmax);
        ymax = __reduce_max_sync(0xffffffffu, ymax);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&bounds[0], xmin);
            atomicMin(&bounds[1], ymin);
            atomicMax(&bounds[2], xmax);
            atomicMax(&bounds[3], ymax);
        }
    }
}

__device__ __forceinline__ bool load_cached(const unsigned long long* vc, int4 tv, TriSetup& o)
{
    // the three records are loaded before any is tested, so that all three
    // loads are in flight together
    const unsigned long long rec[3] = {vc[tv.x], vc[tv.y], vc[tv.z]};
    const int vids[3] = {tv.x, tv.y, tv.z};
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const unsigned long long r = rec[k];
        const int xs = (int16_t)(uint16_t)(r & 0xFFFFu);
        ok = ok && xs != kCulledX;
        o.x[k] = xs;
        o.y[k] = (int16_t)(uint16_t)((r >> 16) & 0xFFFFu);
        o.iz[k] = __uint_as_float((uint32_t)(r >> 32));
        o.vid[k] = vids[k];
    }
    return ok;
}

// Triangle t (its vertex ids tv) loaded at pose P: from the vertex cache, or
// transformed and snapped here.  False if culled.
template <bool VC>
__device__ __forceinline__ bool load_tri(const DevScene& sc, const DevMesh& m, const float* P,
                                         const unsigned long long* vc, int4 tv, TriSetup& o)
{
    if (VC) return load_cached(vc, tv, o);
    return load_triangle(sc, m, P, tv, o);
}

// Full set-up of triangle t at pose P: load, then orientation.  False if
// culled or degenerate.
template <bool VC>
__device__ __forceinline__ bool get_triangle(const DevScene& sc, const DevMesh& m, const float* P,
                                             const unsigned long long* vc, int t, TriSetup& o)
{
    return load_tri<VC>(sc, m, P, vc, __ldg(&m.tris[t]), o) && orient_triangle(o);
}

// n / d for 0 <= n < 2^24 and 1 <= d < 2^24 without an integer division: a
// binary32 estimate (both operands exact, error below one) corrected once.
__device__ __forceinline__ int div_small(int n, int d)
{
    int q = __float2int_rz(__fmul_rn(__int2float_rn(n), __frcp_rn(__int2float_rn(d))));
    const int r = n - q * d;
    q += (r >= d) - (r < 0);
    return q;
}

// Coverage (edge functions and the ownership rule), depth and the z-buffer
// update of sample (u, v) of a set-up triangle (vertices in 1/16 px, 1/Z,
// doubled area A > 0, owns bits per edge), in the tile at (tu0, tv0).
template <bool K32>
__device__ __forceinline__ void raster_sample(const int* x, const int* y, const float* iz, int A, int owns_bits,
                                              int tri, int u, int v, uint32_t* zbuf, int tu0, int tv0, int tw,
                                              int tcap, float izmax, int* err)
{
    const int idx = (v - tv0) * tw + (u - tu0);
    if (!PERCH_CHECKED((unsigned)idx < (unsigned)tcap, err)) return;
    // Early out for a sample that cannot beat the depth already stored here:
    // its depth is at least 1e4 / max(1/Z) less a few 2^-24 relative, so if
    // max(1/Z) (d_here + 2) < 9999 its depth is at least d_here + 2 and its
    // key is larger.  The stored key only decreases, so reading it while other
    // samples update it can only make this test skip less.
    {
        unsigned dh;
        if (K32) {
            const uint32_t w = zbuf[idx];
            dh = w == 0xFFFFFFFFu ? 0xFFFFFFFFu : (w >> 16);
        } else {
            const unsigned long long w = reinterpret_cast<const unsigned long long*>(zbuf)[idx];
            dh = w == kEmptyKey ? 0xFFFFFFFFu : (unsigned)(w >> 32);
        }
        if (dh < 0xFFFFFFF0u && __fmul_rn(izmax, __uint2float_rn(dh + 2u)) < 9999.0f) return;
    }
    const int sx = 16 * u, sy = 16 * v;
    const int w0 = edge_fn(x[1], y[1], x[2], y[2], sx, sy);
    const int w1 = edge_fn(x[2], y[2], x[0], y[0], sx, sy);
    const int w2 = edge_fn(x[0], y[0], x[1], y[1], sx, sy);
    const bool cov = (w0 > 0 || (w0 == 0 && (owns_bits & 1))) &&
                     (w1 > 0 || (w1 == 0 && (owns_bits & 2))) &&
                     (w2 > 0 || (w2 == 0 && (owns_bits & 4)));
    unsigned d;
    if (cov && sample_depth(w0, w1, w2, iz, A, d)) zmin<K32>(zbuf, idx, d, tri, err);
}

// Coverage, depth and the z-buffer update of sample (u, v) of a staged
// triangle: the same tests as raster_sample from the edge coefficients (no
// vertex differences per sample), coverage first so that an uncovered sample
// reads no z-buffer word.
template <bool K32>
__device__ __forceinline__ void raster_staged(const TriStage& e, int u, int v, uint32_t* zbuf, int tu0, int tv0,
                                              int tw, int tcap, int* err)
{
    const int t0 = (int)((unsigned)e.a[0] * (unsigned)u + (unsigned)e.b[0] * (unsigned)v + (unsigned)e.c[0]);
    const int t1 = (int)((unsigned)e.a[1] * (unsigned)u + (unsigned)e.b[1] * (unsigned)v + (unsigned)e.c[1]);
    const int t2 = (int)((unsigned)e.a[2] * (unsigned)u + (unsigned)e.b[2] * (unsigned)v + (unsigned)e.c[2]);
    if ((t0 | t1 | t2) < 0) return;
    const int idx = (v - tv0) * tw + (u - tu0);
    if (!PERCH_CHECKED((unsigned)idx < (unsigned)tcap, err)) return;
    {   // the early out of raster_sample
        const float izmax = fmaxf(e.iz[0], fmaxf(e.iz[1], e.iz[2]));
        unsigned dh;
        if (K32) {
            const uint32_t w = zbuf[idx];
            dh = w == 0xFFFFFFFFu ? 0xFFFFFFFFu : (w >> 16);
        } else {
            const unsigned long long w = reinterpret_cast<const unsigned long long*>(zbuf)[idx];
            dh = w == kEmptyKey ? 0xFFFFFFFFu : (unsigned)(w >> 32);
        }
        if (dh < 0xFFFFFFF0u && __fmul_rn(izmax, __uint2float_rn(dh + 2u)) < 9999.0f) return;
    }
    const int bias = e.bw_bias >> 16;
    unsigned d;
    if (sample_depth(t0 + (bias & 1), t1 + ((bias >> 1) & 1), t2 + (bias >> 2), e.iz, e.A, d))
        zmin<K32>(zbuf, idx, d, e.tri, err);
}

// Rasterise every triangle of mesh m at pose P into the z-buffer tile
// [tu0,tu1) x [tv0,tv1) (row pitch tw).  A warp sets up 32 triangles (one per
// lane); a triangle with one sample in its box is tested in its own lane, the
// others are staged in shared memory (TS, 32 entries per warp) and the
// samples of their boxes spread evenly over the lanes (a prefix sum of the box
// areas, then a binary search per sample for its triangle).  No barrier inside.
//
// LIST: the triangles are list[0 .. n_list) (the tile's bin, written by this
// block) instead of the whole mesh.
template <int NT, bool K32, bool VC, bool LIST = false>
__device__ __forceinline__ void raster_tile(const DevScene& sc, const DevMesh& mesh, const float* P,
                                            const unsigned long long* vc, TriStage* TS, uint32_t* zbuf,
                                            int tu0, int tv0, int tu1, int tv1, int tw, int* err,
                                            const int* list = nullptr, int n_list = 0)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tcap = tw * (tv1 - tv0);
    const int n = LIST ? n_list : mesh.n_tris;
    // id and vertex ids of the lane's next triangle, loaded one iteration ahead
    int t_next = warp * 32 + lane;
    if (LIST && t_next < n) t_next = list[t_next];
    int4 tv_next = warp * 32 + lane < n ? __ldg(&mesh.tris[t_next]) : make_int4(0, 0, 0, 0);
    for (int base = warp * 32; base < n; base += NT) {
        const int i = base + lane;
        const int t = LIST ? t_next : i;
        const int4 tv = tv_next;
        if (i + NT < n) {
            t_next = LIST ? list[i + NT] : i + NT;
            tv_next = __ldg(&mesh.tris[t_next]);
        }
        int area = 0;
        TriSetup o;
        // the sample box does not depend on the orientation: test it first, so
        // that the many triangles covering no sample of the tile skip the rest
        if (i < n && load_tri<VC>(sc, mesh, P, vc, tv, o)) {
            int xmin = min(o.x[0], min(o.x[1], o.x[2])), xmax = max(o.x[0], max(o.x[1], o.x[2]));
            int ymin = min(o.y[0], min(o.y[1], o.y[2])), ymax = max(o.y[0], max(o.y[1], o.y[2]));
            int u0 = max(ceil16(xmin), tu0), u1 = min(floor16(xmax), tu1 - 1);
            int v0 = max(ceil16(ymin), tv0), v1 = min(floor16(ymax), tv1 - 1);
            if (u0 <= u1 && v0 <= v1 && orient_triangle(o)) {
                const int owns_bits = (owns(o.x[2] - o.x[1], o.y[2] - o.y[1]) ? 1 : 0) |
                                      (owns(o.x[0] - o.x[2], o.y[0] - o.y[2]) ? 2 : 0) |
                                      (owns(o.x[1] - o.x[0], o.y[1] - o.y[0]) ? 4 : 0);
                const float izmax = fmaxf(o.iz[0], fmaxf(o.iz[1], o.iz[2]));
                if (u0 == u1 && v0 == v1) {
                    // one sample in the box (most triangles of a fine mesh):
                    // test it in this lane, no staging
                    raster_sample<K32>(o.x, o.y, o.iz, o.A, owns_bits, t, u0, v0, zbuf, tu0, tv0, tw, tcap, izmax,
                                       err);
                } else {
                    area = (u1 - u0 + 1) * (v1 - v0 + 1);
                    // edge i from vertex p to vertex q at the sample (16 u, 16 v):
                    // (xq - xp)(16 v - yp) - (yq - yp)(16 u - xp), less its tie bias
                    TriStage e;
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const int p = (i + 1) % 3, q = (i + 2) % 3;
                        const unsigned dx = (unsigned)o.x[q] - (unsigned)o.x[p];
                        const unsigned dy = (unsigned)o.y[q] - (unsigned)o.y[p];
                        e.a[i] = (int)(0u - 16u * dy);
                        e.b[i] = (int)(16u * dx);
                        e.c[i] = (int)(dy * (unsigned)o.x[p] - dx * (unsigned)o.y[p] - (unsigned)(((owns_bits >> i) & 1) ^ 1));
                        e.iz[i] = o.iz[i];
                    }
                    e.A = o.A;
                    e.tri = t;
                    e.uv0 = u0 | (v0 << 16);
                    e.bw_bias = (u1 - u0 + 1) | ((~owns_bits & 7) << 16);
                    TS[lane] = e;                  // whole-record store
                }
            }
        }
        // the larger boxes: their samples spread evenly over the lanes
        if (__ballot_sync(0xffffffffu, area > 0) == 0u) continue;
        int incl = area;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int x = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += x;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        __syncwarp();
        for (int f0 = 0; f0 < total; f0 += 32) {
            const int f = f0 + lane;
            // the triangle j whose pixel range holds f: incl[j-1] <= f < incl[j]
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                int v = __shfl_sync(0xffffffffu, incl, j + step - 1);
                if (v <= f) j += step;
            }
            const int excl = __shfl_sync(0xffffffffu, incl, j > 0 ? j - 1 : 0);
            if (f >= total) continue;
            const TriStage e = TS[j];              // whole-record load
            const int local = f - (j > 0 ? excl : 0);
            const int bw = e.bw_bias & 0xFFFF;
            const int dv = div_small(local, bw);
            raster_staged<K32>(e, (e.uv0 & 0xFFFF) + (local - dv * bw), (e.uv0 >> 16) + dv, zbuf, tu0, tv0, tw, tcap,
                               err);
        }
        __syncwarp();
    }
}

// Tile bins of one hypothesis: the pixel box rbox is rasterised in tiles of tw
// x th pixels (n_tx per row of tiles); every triangle whose sample box meets a
// tile is listed in that tile's bin (bins + tile * cap, count in cnt[tile];
// a count above cap marks a bin that overflowed).  A triangle covers samples
// only inside its sample box, so a tile rasterised from its bin gets the same
// z-buffer as from the whole mesh.  Bin order depends on timing; the
// z-buffer does not (atomicMin).
template <int NT, bool VC>
__device__ void bin_triangles(const DevScene& sc, const DevMesh& mesh, const float* P, const unsigned long long* vc,
                              const int* rbox, int tw, int th, int n_tx, int* bins, int cap, int* cnt)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int4 tv_next = warp * 32 + lane < mesh.n_tris ? __ldg(&mesh.tris[warp * 32 + lane]) : make_int4(0, 0, 0, 0);
    for (int base = warp * 32; base < mesh.n_tris; base += NT) {
        const int t = base + lane;
        const int4 tv = tv_next;
        if (t + NT < mesh.n_tris) tv_next = __ldg(&mesh.tris[t + NT]);
        TriSetup o;
        if (t >= mesh.n_tris || !load_tri<VC>(sc, mesh, P, vc, tv, o)) continue;
        const int u0 = max(ceil16(min(o.x[0], min(o.x[1], o.x[2]))), rbox[0]);
        const int u1 = min(floor16(max(o.x[0], max(o.x[1], o.x[2]))), rbox[2] - 1);
        const int v0 = max(ceil16(min(o.y[0], min(o.y[1], o.y[2]))), rbox[1]);
        const int v1 = min(floor16(max(o.y[0], max(o.y[1], o.y[2]))), rbox[3] - 1);
        if (u0 > u1 || v0 > v1) continue;
        const int tx0 = div_small(u0 - rbox[0], tw), tx1 = div_small(u1 - rbox[0], tw);
        const int ty0 = div_small(v0 - rbox[1], th), ty1 = div_small(v1 - rbox[1], th);
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                const int tile = ty * n_tx + tx;
                const int k = atomicAdd(&cnt[tile], 1);
                if (k < cap) bins[tile * cap + k] = t;
            }
    }
}

// Affine integer colour at pixel (u, v) of the set-up triangle o: per channel
// (w0 c0 + w1 c1 + w2 c2 + floor(A / 2)) / A with the edge values w of the
// pixel's sample (screen-space interpolation of the per-vertex colour, rounded
// half up), packed r | g << 8 | b << 16.
__device__ __forceinline__ uint32_t interp_colour(const DevMesh& m, const TriSetup& o, int u, int v)
{
    const int sx = 16 * u, sy = 16 * v;
    const long long w0 = edge_fn(o.x[1], o.y[1], o.x[2], o.y[2], sx, sy);
    const long long w1 = edge_fn(o.x[2], o.y[2], o.x[0], o.y[0], sx, sy);
    const long long w2 = edge_fn(o.x[0], o.y[0], o.x[1], o.y[1], sx, sy);
    const uint32_t c0 = __float_as_uint(__ldg(&m.verts[o.vid[0]].w));
    const uint32_t c1 = __float_as_uint(__ldg(&m.verts[o.vid[1]].w));
    const uint32_t c2 = __float_as_uint(__ldg(&m.verts[o.vid[2]].w));
    const long long half = o.A / 2;
    // floor(num / A) without a 64-bit division: a binary32 estimate from the
    // reciprocal of A (relative error a few 2^-24, and the quotient is below
    // 256, so the estimate is off by at most one) corrected exactly with
    // integer arithmetic
    const float rA = __frcp_rn(__int2float_rn(o.A));
    uint32_t crgb = 0;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const long long num = w0 * ((c0 >> (8 * ch)) & 255) + w1 * ((c1 >> (8 * ch)) & 255) +
                              w2 * ((c2 >> (8 * ch)) & 255) + half;
        // num < 2^41: its binary32 value from two 32-bit halves (the
        // estimate needs only relative accuracy, the correction makes it exact)
        const float numf = __fadd_rn(__fmul_rn(__int2float_rn((int)(num >> 16)), 65536.0f),
                                     __int2float_rn((int)(num & 0xFFFF)));
        long long q = __float2int_rz(__fmul_rn(numf, rA));
        const long long r = num - q * o.A;
        q += (r >= o.A) - (r < 0);
        crgb |= (uint32_t)q << (8 * ch);
    }
    return crgb;
}

// jo_mode 1 with the colour check (Eq. 3 with Eq. 4 applied from the observed
// side): every observed point p of rows [mv0, mv1) of the admissible box
// holds the key of its nearest rendered point q; p stays an inlier iff the
// CIEDE2000 difference between q's rendered colour and p's colour is at most
// tau_c, else its key is cleared.  This handles the p whose q lies in the
// z-buffer tile [tu0, tu1) x [tv0, tv1) now in shared memory (q's winning
// triangle gives its colour).
template <int NT, bool K32, bool VC>
__device__ __forceinline__ void jo_colour_pass(const Job& J, const float* P, const unsigned long long* vc, const ScoreSmem& S,
                               int tu0, int tv0, int tu1, int tv1, int tw, const int* vbox, int mv0, int mv1)
{
    const DevScene& sc = J.sc;
    const int vw = vbox[2] - vbox[0];
    const int n = vw * (mv1 - mv0);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(S.marks);
    for (int i = threadIdx.x; i < n; i += NT) {
        const unsigned long long k = keys[i];
        if (k == kEmptyKey) continue;
        const uint32_t qp = (uint32_t)k;
        const int qu = (int)(qp & 0xFFFFu), qv = (int)(qp >> 16);
        if (qu < tu0 || qu >= tu1 || qv < tv0 || qv >= tv1) continue;
        const int zi = (qv - tv0) * tw + (qu - tu0);
        // q is a kept rendered point: its z-buffer word holds its triangle
        const int tri = K32 ? (int)(S.zbuf[zi] & 0xFFFFu)
                            : (int)(uint32_t)reinterpret_cast<const unsigned long long*>(S.zbuf)[zi];
        TriSetup o;
        get_triangle<VC>(sc, J.m, P, vc, tri, o);
        const uint32_t crgb = interp_colour(J.m, o, qu, qv);
        const int pu = vbox[0] + i % vw, pv = mv0 + i / vw;
        const float4 lp = __ldg(&sc.lab[pv * sc.W + pu]);
        const float3 lq = srgb8_to_lab(crgb & 255, (crgb >> 8) & 255, (crgb >> 16) & 255);
        if (ciede2000(lq, make_float3(lp.x, lp.y, lp.z)) > sc.tau_c) keys[i] = kEmptyKey;
    }
}

// Specialisations of the scoring kernel: plain scoring (jo_mode 0), edges of
// the Monotone Scene Generation tree, and jo_mode 1 (Eq. 3 as written, with
// per-pixel nearest-rendered-point keys).  Each is compiled separately so the
// plain path carries none of the other two's code.
enum : int { kModePlain = 0, kModeTree = 1, kModeEq3 = 2 };

// Is the observed point p of pixel pix in the admissible set V(O) at pose P
// (Sec. IV-A J_o; labels Sec. V-C)?  The inscribed cylinder about the
// object's z-axis (radius^2 rr, height vol_h) in the object frame, R^T (p - t),
// or the pixel's label.
__device__ __forceinline__ bool in_admissible(const DevScene& sc, const Job& J, const float* P, float rr, int pix,
                                              float4 p)
{
    if (J.label >= 0) return __ldg(&sc.labels[pix]) == J.label;
    float e0 = __fsub_rn(p.x, P[3]), e1 = __fsub_rn(p.y, P[7]), e2 = __fsub_rn(p.z, P[11]);
    float q0 = __fadd_rn(__fadd_rn(__fmul_rn(P[0], e0), __fmul_rn(P[4], e1)), __fmul_rn(P[8], e2));
    float q1 = __fadd_rn(__fadd_rn(__fmul_rn(P[1], e0), __fmul_rn(P[5], e1)), __fmul_rn(P[9], e2));
    float q2 = __fadd_rn(__fadd_rn(__fmul_rn(P[2], e0), __fmul_rn(P[6], e1)), __fmul_rn(P[10], e2));
    return __fadd_rn(__fmul_rn(q0, q0), __fmul_rn(q1, q1)) <= rr && q2 >= 0.0f && q2 <= J.m.vol_h;
}

// |I cap V| of plain scoring, counted in chunks of kJoChunk lattice pixels of
// the whole admissible box taken from a shared counter (zero at the start of
// the hypothesis).  It needs nothing rendered, so warps that finish the
// raster early count chunks while the others still rasterise (`stop`: the
// count of warps done with the raster; they stop once all are), and the
// chunks left over are counted after the search.
constexpr int kJoChunk = 256;

template <int NT>
__device__ void jo_count_in(const DevScene& sc, const Job& J, const float* P, const int* vbox, int* counter,
                            const int* stop, int& n_in)
{
    const int s = sc.stride, lane = threadIdx.x & 31;
    const int us0 = ((vbox[0] + s - 1) / s) * s, vs0 = ((vbox[1] + s - 1) / s) * s;
    const int nu = us0 < vbox[2] ? (vbox[2] - 1 - us0) / s + 1 : 0;
    const int nv = vs0 < vbox[3] ? (vbox[3] - 1 - vs0) / s + 1 : 0;
    const int npx = nu * nv;
    const float rr = __fmul_rn(J.m.vol_r, J.m.vol_r);
    for (;;) {
        if (stop && *reinterpret_cast<const volatile int*>(stop) >= NT / 32) break;
        int c = 0;
        if (lane == 0) c = atomicAdd(counter, 1);
        const int k0 = __shfl_sync(0xffffffffu, c, 0) * kJoChunk;
        if (k0 >= npx) break;
        const int k1 = min(k0 + kJoChunk, npx);
        for (int k = k0 + lane; k < k1; k += 32) {
            const int kv = div_small(k, nu);
            const int pix = (vs0 + kv * s) * sc.W + us0 + (k - kv * nu) * s;
            const float4 p = __ldg(&sc.pxyz[pix]);
            if (p.w != 0.0f && in_admissible(sc, J, P, rr, pix, p)) ++n_in;
        }
    }
}

// Rasterise, resolve and radius-search the pixel box rbox in z-buffer tiles.
// J_r is accumulated when count_jr; marks are set for nearest neighbours that
// fall in rows [mv0, mv1) of the admissible box vbox.
template <int NT, bool K32, bool VC, int MODE, bool BINS>
__device__ void score_tiles(const ScoreArgs& a, const Job& J, const float* P, const unsigned long long* vc,
                            const int* rbox, const ScoreSmem& S, const int* vbox, int mv0, int mv1,
                            bool count_jr, int& jr_local, int& n_in, int& n_marked)
{
    constexpr bool TREE = MODE == kModeTree, EQ3 = MODE == kModeEq3;
    const DevScene& sc = J.sc;
    const float rr = __fmul_rn(J.m.vol_r, J.m.vol_r);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpProbe& WP = *reinterpret_cast<WarpProbe*>(reinterpret_cast<char*>(S.probe) + warp * kWarpScratch);
    TriStage* TS = reinterpret_cast<TriStage*>(reinterpret_cast<char*>(S.stage) + warp * kWarpScratch);
    const int s = sc.stride;
    const int rw = rbox[2] - rbox[0], rh = rbox[3] - rbox[1];
    if (rw <= 0 || rh <= 0) return;
    const int cap_px = K32 ? a.zcap_words : a.zcap_words / 2;
    const int tw = min(rw, cap_px);
    const int th = max(1, cap_px / tw);
    const uint32_t empty32 = 0xFFFFFFFFu;
    const int vw = vbox[2] - vbox[0];
    uint32_t* zbuf = S.zbuf;
    // a pixel box of several tiles: each tile's triangles binned first
    const int n_tx = (rw + tw - 1) / tw, n_tiles = n_tx * ((rh + th - 1) / th);
    const bool binned = BINS && VC && a.bin_cap > 0 && n_tiles > 1 && n_tiles <= kBinTiles;
    int* bins = binned ? reinterpret_cast<int*>(const_cast<unsigned long long*>(vc) + a.bin_off) : nullptr;
    if (binned) {
        for (int i = threadIdx.x; i < n_tiles; i += NT) S.bin_cnt[i] = 0;
        __syncthreads();
        if (BINS) bin_triangles<NT, VC>(sc, J.m, P, vc, rbox, tw, th, n_tx, bins, a.bin_cap, S.bin_cnt);
        __syncthreads();
    }
    int tile = 0;
    for (int tv0 = rbox[1]; tv0 < rbox[3]; tv0 += th) {
        for (int tu0 = rbox[0]; tu0 < rbox[2]; tu0 += tw, ++tile) {
            const int tu1 = min(tu0 + tw, rbox[2]), tv1 = min(tv0 + th, rbox[3]);
            const int tpx = tw * (tv1 - tv0);
            const int words = K32 ? tpx : 2 * tpx;
            for (int i = threadIdx.x; i < words; i += NT) zbuf[i] = empty32;
            if (threadIdx.x == 0) {
                *S.next_batch = 0;
                *S.raster_done = 0;
            }
            __syncthreads();
            if (BINS && binned && S.bin_cnt[tile] <= a.bin_cap)
                raster_tile<NT, K32, VC, BINS>(sc, J.m, P, vc, TS, zbuf, tu0, tv0, tu1, tv1, tw, a.err,
                                               bins + tile * a.bin_cap, S.bin_cnt[tile]);
            else
                raster_tile<NT, K32, VC>(sc, J.m, P, vc, TS, zbuf, tu0, tv0, tu1, tv1, tw, a.err);
            if (MODE == kModePlain && count_jr) {
                // the raster's early finishers count J_o's |I cap V| meanwhile
                if (lane == 0) atomicAdd(S.raster_done, 1);
                __syncwarp();
                jo_count_in<NT>(sc, J, P, vbox, S.jo_next, S.raster_done, n_in);
            }
            __syncthreads();
            if (a.dump) {
                for (int i = threadIdx.x; i < tpx; i += NT) {
                    int u = tu0 + i % tw, v = tv0 + i / tw;
                    if (u >= tu1) continue;
                    unsigned long long k;
                    if (K32) {
                        uint32_t w = zbuf[i];
                        k = (w == empty32) ? kEmptyKey
                                           : (((unsigned long long)(w >> 16) << 32) | (w & 0xFFFFu));
                    } else {
                        k = reinterpret_cast<unsigned long long*>(zbuf)[i];
                    }
                    a.dump[(size_t)v * sc.W + u] = k;
                }
            }
            // ---- resolve + radius search.  The stride lattice of the tile is
            // cut into 8 x 4 pixel blocks that warps take from a counter; a
            // warp resolves a block (occluder test, colour, back-projection)
            // and appends its kept points to its own queue, which it searches
            // 32 at a time -- no block-wide barrier until the tile is done.
            const int us0 = ((tu0 + s - 1) / s) * s, vs0 = ((tv0 + s - 1) / s) * s;
            const int nu = us0 < tu1 ? (tu1 - 1 - us0) / s + 1 : 0;
            const int nv = vs0 < tv1 ? (tv1 - 1 - vs0) / s + 1 : 0;
            const int nbx = (nu + 7) / 8, nby = (nv + 3) / 4;
            const int nblocks = nbx * nby;
            KeptPoint* wq = S.kept + warp * kWarpQueue;
            const MarkBand mband = {S.marks, vbox[0], vbox[2], mv0, mv1, vw, a.err};
            __syncwarp();
            int wq_head = 0, wq_count = 0;
            for (;;) {
                int blk = 0;
                if (lane == 0) blk = atomicAdd(S.next_batch, 1);
                blk = __shfl_sync(0xffffffffu, blk, 0);
                const bool more = blk < nblocks;
                if (more) {
                    bool kept = false;
                    KeptPoint kp;
                    const int by = div_small(blk, nbx);
                    const int lu = (blk - by * nbx) * 8 + (lane & 7), lv = by * 4 + (lane >> 3);
                    if (lu < nu && lv < nv) {
                        int u = us0 + lu * s, v = vs0 + lv * s;
                        int zi = (v - tv0) * tw + (u - tu0);
                        unsigned d = 0;
                        int tri = -1;
                        if (!PERCH_CHECKED((unsigned)zi < (unsigned)(tw * (tv1 - tv0)), a.err)) {
                        } else if (K32) {
                            uint32_t w = zbuf[zi];
                            if (w != empty32) { d = w >> 16; tri = (int)(w & 0xFFFFu); }
                        } else {
                            unsigned long long w = reinterpret_cast<unsigned long long*>(zbuf)[zi];
                            if (w != kEmptyKey) { d = (unsigned)(w >> 32); tri = (int)(uint32_t)w; }
                        }
                        int pix = v * sc.W + u;
                        if (TREE && tri >= 0) {
                            // a placed object in front hides the pixel; one behind
                            // by more than the margin refuses the edge
                            const unsigned sd = __ldg(&J.tree.depth[pix]);
                            if (sd != 0) {
                                if ((unsigned long long)d + (unsigned)J.tree.margin < sd) *S.refused = 1;
                                if (!(d < sd)) tri = -1;
                            }
                            if (tri >= 0 && J.tree.out_depth) J.tree.out_depth[pix] = d;
                        }
                        if (tri >= 0) {
                            unsigned dobs = __ldg(&sc.depth[pix]);
                            bool occluded = sc.occ_margin >= 0 && dobs > 0 &&
                                            (unsigned long long)dobs + (unsigned)sc.occ_margin < d &&
                                            (J.label < 0 || __ldg(&sc.labels[pix]) != J.label);
                            if (!occluded) {
                                float3 q = back_project(sc, u, v, d);
                                kp.x = q.x; kp.y = q.y; kp.z = q.z; kp.pix = (uint32_t)u | ((uint32_t)v << 16);
                                kept = true;
                                if (sc.near_bits) {
                                    // no observed point in the 27 cells: unexplained
                                    // without a search (the radius search's own filter)
                                    const long long b = near_index(sc, cell_coord(q.x, sc.inv_cell),
                                                                   cell_coord(q.y, sc.inv_cell),
                                                                   cell_coord(q.z, sc.inv_cell));
                                    if (b < 0 || !((__ldg(&sc.near_bits[b >> 5]) >> (b & 31)) & 1u)) {
                                        kept = false;
                                        if (count_jr) ++jr_local;
                                    }
                                }
                            }
                        }
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, kept);
                    if (kept) wq[(wq_head + wq_count + __popc(bal & ((1u << lane) - 1u))) % kWarpQueue] = kp;
                    wq_count += __popc(bal);
                }
                // search a full batch, or what is left once the blocks run out
                while (wq_count >= 32 || (!more && wq_count > 0)) {
                    __syncwarp();
                    const int nb = min(wq_count, 32);
                    const bool valid = lane < nb;
                    KeptPoint kq = {0.f, 0.f, 0.f, 0u};
                    if (valid) kq = wq[(wq_head + lane) % kWarpQueue];
                    wq_head = (wq_head + nb) % kWarpQueue;
                    wq_count -= nb;
                    const uint32_t qpix = (EQ3 && valid) ? kq.pix : 0u;
                    const unsigned long long nn = probe_batch<EQ3>(sc, valid, kq.x, kq.y, kq.z, qpix, WP, lane, mband);
                    if (valid) {
                        bool explained = nn != kEmptyKey;
                        const int pnn = (int)(uint32_t)nn;
                        const int pu = pnn & 0xFFFF, pv = pnn >> 16;
                        if (explained && sc.color_check) {
                            // the rendered colour of q, from the triangle its z-buffer word holds
                            const int qu = (int)(kq.pix & 0xFFFFu), qv = (int)(kq.pix >> 16);
                            const int qi = (qv - tv0) * tw + (qu - tu0);
                            const int qtri = K32 ? (int)(zbuf[qi] & 0xFFFFu)
                                                 : (int)(uint32_t)reinterpret_cast<const unsigned long long*>(zbuf)[qi];
                            TriSetup o;
                            get_triangle<VC>(sc, J.m, P, vc, qtri, o);
                            const uint32_t rgb = interp_colour(J.m, o, qu, qv);
                            float4 lp = __ldg(&sc.lab[pv * sc.W + pu]);
                            float3 lq = srgb8_to_lab(rgb & 255, (rgb >> 8) & 255, (rgb >> 16) & 255);
                            if (ciede2000(lq, make_float3(lp.x, lp.y, lp.z)) > sc.tau_c) explained = false;
                        }
                        if (TREE && explained && J.tree.out_mark) {
                            const int npix = pv * sc.W + pu;
                            atomicOr(&J.tree.out_mark[npix >> 5], 1u << (npix & 31));
                        }
                        if (!explained) {
                            if (count_jr) ++jr_local;
                        } else if (!EQ3) {
                            if (pu >= vbox[0] && pu < vbox[2] && pv >= mv0 && pv < mv1) {
                                int bit = (pv - mv0) * vw + (pu - vbox[0]);
                                if (PERCH_CHECKED((unsigned)bit < 32u * (unsigned)a.mark_words, a.err)) {
                                    const unsigned m = 1u << (bit & 31);
                                    const unsigned was = atomicOr(&S.marks[bit >> 5], m);
                                    if (MODE == kModePlain && !(was & m)) {
                                        // J_o's marked part: the first mark of a pixel of V
                                        const int npix = pv * sc.W + pu;
                                        const float4 pn = __ldg(&sc.pxyz[npix]);
                                        if (pn.w != 0.0f && in_admissible(sc, J, P, rr, npix, pn)) ++n_marked;
                                    }
                                }
                            }
                        }
                    }
                }
                if (!more) break;
            }
            __syncthreads();
            if (threadIdx.x == 0) *S.next_batch = 0;
            __syncthreads();
        }
    }
}

// jo_mode 1 with the colour check, after score_tiles has made every key of
// the band final: the colour pass over the same z-buffer tiles.  With one
// tile its z-buffer is still in shared memory; otherwise each tile is
// rendered again.
template <int NT, bool K32, bool VC>
__device__ __noinline__ void jo_colour_band(const ScoreArgs& a, const Job& J, const float* P,
                                            const unsigned long long* vc, const int* rbox, const ScoreSmem& S,
                                            const int* vbox, int mv0, int mv1)
{
    const int warp = threadIdx.x >> 5;
    TriStage* TS = reinterpret_cast<TriStage*>(reinterpret_cast<char*>(S.stage) + warp * kWarpScratch);
    const int rw = rbox[2] - rbox[0], rh = rbox[3] - rbox[1];
    if (rw <= 0 || rh <= 0) return;
    const int cap_px = K32 ? a.zcap_words : a.zcap_words / 2;
    const int tw = min(rw, cap_px);
    const int th = max(1, cap_px / tw);
    if (th >= rh) {
        jo_colour_pass<NT, K32, VC>(J, P, vc, S, rbox[0], rbox[1], rbox[2], rbox[3], tw, vbox, mv0, mv1);
        __syncthreads();
        return;
    }
    for (int tv0 = rbox[1]; tv0 < rbox[3]; tv0 += th) {
        for (int tu0 = rbox[0]; tu0 < rbox[2]; tu0 += tw) {
            const int tu1 = min(tu0 + tw, rbox[2]), tv1 = min(tv0 + th, rbox[3]);
            const int words = K32 ? tw * (tv1 - tv0) : 2 * tw * (tv1 - tv0);
            for (int i = threadIdx.x; i < words; i += NT) S.zbuf[i] = 0xFFFFFFFFu;
            __syncthreads();
            raster_tile<NT, K32, VC>(J.sc, J.m, P, vc, TS, S.zbuf, tu0, tv0, tu1, tv1, tw, a.err);
            __syncthreads();
            jo_colour_pass<NT, K32, VC>(J, P, vc, S, tu0, tv0, tu1, tv1, tw, vbox, mv0, mv1);
            __syncthreads();
        }
    }
}

// Score hypothesis h (one block).  Writes costs[2h] = J_o, costs[2h+1] = J_r.
template <int NT, int MODE, bool BINS>
__device__ void score_one(const ScoreArgs& a, const Job& J, long long h, const ScoreSmem& S, float* s_pose,
                          int* s_rbox, int* s_vbox, int* s_k32, int (*s_red)[NT / 32],
                          unsigned long long* vc)
{
    constexpr bool TREE = MODE == kModeTree;
    const DevScene& sc = J.sc;
    if (threadIdx.x < 12) s_pose[threadIdx.x] = J.poses[h * 12 + threadIdx.x];
    if (TREE && threadIdx.x == 0) *S.refused = 0;
    if (threadIdx.x == 0) *S.jo_next = 0;
    if (threadIdx.x < 4) S.vbounds[threadIdx.x] = threadIdx.x < 2 ? INT_MAX : INT_MIN;
    __syncthreads();
    // the two boxes in two warps, in parallel with each other and with the
    // other warps' share of the vertex pass
    if (threadIdx.x == 0) {
        float zmax;
        project_box(sc, s_pose, J.m.lo, J.m.hi, J.roi[0], J.roi[1], J.roi[2], J.roi[3], s_rbox, &zmax);
        *s_k32 = (J.m.n_tris <= 65535 && zmax < 6.5f) ? 1 : 0;
    } else if (threadIdx.x == 32) {
        if (J.label >= 0) {
            s_vbox[0] = J.roi[0]; s_vbox[1] = J.roi[1]; s_vbox[2] = J.roi[2]; s_vbox[3] = J.roi[3];
        } else {
            float lo[3] = {-J.m.vol_r, -J.m.vol_r, 0.0f}, hi[3] = {J.m.vol_r, J.m.vol_r, J.m.vol_h};
            float zv;
            project_box(sc, s_pose, lo, hi, 0, 0, sc.W, sc.H, s_vbox, &zv);
        }
    }
    const bool use_vc = vc != nullptr;
    if (use_vc) vertex_pass(sc, J.m, s_pose, vc, NT, S.vbounds);
    __syncthreads();
    // The pixel box of the render: the projected object-frame box, tightened
    // (with the vertex cache) to the samples between the kept vertices'
    // smallest and largest snapped coordinates -- every covered sample lies
    // in its triangle's vertex box, so nothing outside can be covered.
    int rb[4] = {s_rbox[0], s_rbox[1], s_rbox[2], s_rbox[3]};
    if (use_vc) {
        const int* vb = S.vbounds;
        if (vb[0] > vb[2]) {
            rb[2] = rb[0];
            rb[3] = rb[1];
        } else {
            rb[0] = max(rb[0], ceil16(vb[0]));
            rb[1] = max(rb[1], ceil16(vb[1]));
            rb[2] = max(rb[0], min(rb[2], floor16(vb[2]) + 1));
            rb[3] = max(rb[1], min(rb[3], floor16(vb[3]) + 1));
        }
    }

    // The admissible box is handled in bands of rows that fit the marks
    // bitset (jo_mode 1: one 64-bit key per pixel); each band repeats the
    // render + search (J_r counted once).
    constexpr bool jo1 = MODE == kModeEq3;
    const int vw = s_vbox[2] - s_vbox[0], vh = s_vbox[3] - s_vbox[1];
    const int band_rows = vw > 0 ? max(1, (jo1 ? a.mark_words / 2 : 32 * a.mark_words) / vw) : 1;
    const int n_bands = vh > 0 ? (vh + band_rows - 1) / band_rows : 1;
    int jr = 0, n_in = 0, n_marked = 0;
    const int s = sc.stride;
    const float* P = s_pose;
    const float rr = __fmul_rn(J.m.vol_r, J.m.vol_r);
    for (int band = 0; band < n_bands; ++band) {
        const int mv0 = s_vbox[1] + band * band_rows;
        const int mv1 = min(mv0 + band_rows, s_vbox[3]);
        const int mwords = jo1 ? 2 * vw * max(0, mv1 - mv0) : (vw * max(0, mv1 - mv0) + 31) / 32;
        const uint32_t mfill = jo1 ? 0xFFFFFFFFu : 0u;     // empty keys / clear bits
        for (int i = threadIdx.x; i < mwords; i += NT) S.marks[i] = mfill;
        __syncthreads();
        if (*s_k32) {
            if (use_vc) score_tiles<NT, true, true, MODE, BINS>(a, J, P, vc, rb, S, s_vbox, mv0, mv1, band == 0, jr,
                                                               n_in, n_marked);
            else score_tiles<NT, true, false, MODE, BINS>(a, J, P, vc, rb, S, s_vbox, mv0, mv1, band == 0, jr,
                                                               n_in, n_marked);
        } else {
            if (use_vc) score_tiles<NT, false, true, MODE, BINS>(a, J, P, vc, rb, S, s_vbox, mv0, mv1, band == 0, jr,
                                                               n_in, n_marked);
            else score_tiles<NT, false, false, MODE, BINS>(a, J, P, vc, rb, S, s_vbox, mv0, mv1, band == 0, jr,
                                                               n_in, n_marked);
        }
        __syncthreads();
        if (jo1 && sc.color_check) {
            // Eq. 4 from the observed side, once the band's keys are final
            if (*s_k32) {
                if (use_vc) jo_colour_band<NT, true, true>(a, J, P, vc, rb, S, s_vbox, mv0, mv1);
                else jo_colour_band<NT, true, false>(a, J, P, vc, rb, S, s_vbox, mv0, mv1);
            } else {
                if (use_vc) jo_colour_band<NT, false, true>(a, J, P, vc, rb, S, s_vbox, mv0, mv1);
                else jo_colour_band<NT, false, false>(a, J, P, vc, rb, S, s_vbox, mv0, mv1);
            }
        }
        // plain scoring: J_o's marked part was counted as the marks were set
        // (each pixel of V once, by the lane whose atomicOr set its bit) and
        // |I cap V| is counted by jo_count_in
        if (MODE == kModePlain) continue;
        // ---- J_o over the admissible set V(h), rows [mv0, mv1)
        const int us0 = ((s_vbox[0] + s - 1) / s) * s, vs0 = ((mv0 + s - 1) / s) * s;
        const int nu = us0 < s_vbox[2] ? (s_vbox[2] - 1 - us0) / s + 1 : 0;
        const int nv = vs0 < mv1 ? (mv1 - 1 - vs0) / s + 1 : 0;
        // pixel k = (row k / nu, column k % nu), the row and column carried
        // from one k to the next (k advances by NT) instead of divided out
        int kr = nu > 0 ? div_small(threadIdx.x, nu) : 0, kc = threadIdx.x - kr * nu;
        const int rstep = nu > 0 ? div_small(NT, nu) : 0, cstep = NT - rstep * nu;
        for (int k = threadIdx.x; k < nu * nv; k += NT) {
            const int u = us0 + kc * s, v = vs0 + kr * s;
            kc += cstep;
            kr += rstep;
            if (kc >= nu) { kc -= nu; ++kr; }
            int pix = v * sc.W + u;
            // the observed point of the pixel, back-projected once per scene
            const float4 p = __ldg(&sc.pxyz[pix]);
            if (p.w == 0.0f) continue;
            bool in;
            if (J.label >= 0) {
                in = __ldg(&sc.labels[pix]) == J.label;
            } else {
                float e0 = __fsub_rn(p.x, P[3]), e1 = __fsub_rn(p.y, P[7]), e2 = __fsub_rn(p.z, P[11]);
                float q0 = __fadd_rn(__fadd_rn(__fmul_rn(P[0], e0), __fmul_rn(P[4], e1)), __fmul_rn(P[8], e2));
                float q1 = __fadd_rn(__fadd_rn(__fmul_rn(P[1], e0), __fmul_rn(P[5], e1)), __fmul_rn(P[9], e2));
                float q2 = __fadd_rn(__fadd_rn(__fmul_rn(P[2], e0), __fmul_rn(P[6], e1)), __fmul_rn(P[10], e2));
                in = __fadd_rn(__fmul_rn(q0, q0), __fmul_rn(q1, q1)) <= rr && q2 >= 0.0f && q2 <= J.m.vol_h;
            }
            if (in) {
                if (TREE) {
                    if (J.tree.out_vol) atomicOr(&J.tree.out_vol[pix >> 5], 1u << (pix & 31));
                    if ((__ldg(&J.tree.vol[pix >> 5]) >> (pix & 31)) & 1u) continue;   // counted before
                }
                ++n_in;
                int bit = (v - mv0) * vw + (u - s_vbox[0]);
                if (!PERCH_CHECKED((unsigned)bit < (jo1 ? (unsigned)a.mark_words / 2u : 32u * (unsigned)a.mark_words), a.err))
                    continue;
                unsigned mk = jo1 ? (reinterpret_cast<const unsigned long long*>(S.marks)[bit] != kEmptyKey)
                                  : (S.marks[bit >> 5] >> (bit & 31)) & 1u;
                if (TREE && !mk) mk = (__ldg(&J.tree.mark[pix >> 5]) >> (pix & 31)) & 1u;
                n_marked += mk;
            }
        }
        __syncthreads();
    }
    // the chunks of |I cap V| the raster's early finishers did not count
    if (MODE == kModePlain) jo_count_in<NT>(sc, J, P, s_vbox, S.jo_next, nullptr, n_in);
    // ---- warp-shuffle reduction of (J_r, |I cap V|, marked)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        jr += __shfl_xor_sync(0xffffffffu, jr, o);
        n_in += __shfl_xor_sync(0xffffffffu, n_in, o);
        n_marked += __shfl_xor_sync(0xffffffffu, n_marked, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_red[0][warp] = jr; s_red[1][warp] = n_in; s_red[2][warp] = n_marked; }
    __syncthreads();
    if (threadIdx.x < 32) {
        int x = lane < NT / 32 ? s_red[0][lane] : 0;
        int y = lane < NT / 32 ? s_red[1][lane] : 0;
        int z = lane < NT / 32 ? s_red[2][lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
            z += __shfl_xor_sync(0xffffffffu, z, o);
        }
        if (lane == 0) {
            const bool refused = TREE && *S.refused;
            J.costs[2 * h] = refused ? -1 : y - z;
            J.costs[2 * h + 1] = refused ? -1 : x;
        }
    }
    __syncthreads();
}

// Byte offsets of the dynamic shared-memory regions of a scoring block; every
// region starts on a 16-byte boundary (the queues and the per-warp scratch
// hold float4 and 64-bit fields).
struct SmemLayout {
    size_t marks, kept, probe, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline SmemLayout smem_layout(int zcap_words, int mark_words, int threads)
{
    SmemLayout L;
    L.marks = align16(sizeof(uint32_t) * (size_t)zcap_words);
    L.kept = align16(L.marks + sizeof(uint32_t) * (size_t)mark_words);
    L.probe = align16(L.kept + sizeof(KeptPoint) * kWarpQueue * (size_t)(threads / 32));
    L.total = align16(L.probe + kWarpScratch * (size_t)(threads / 32));
    return L;
}

// Claim one vertex-cache slot from a pool of nslots (bit set = in use).
// Blocks of every scoring kernel that runs at the same time with the same
// launch shape draw from one pool sized for the device's resident blocks, so
// a free slot exists; should none be found the block runs without the cache
// (same results).  Bounded: every failed attempt adds a bit to `seen`.
__device__ int claim_vslot(unsigned* mask, int nslots)
{
    const int words = (nslots + 31) >> 5;
    for (int k = 0; k < words; ++k) {
        const int w = (int)((blockIdx.x + k) % words);
        const int rem = nslots - 32 * w;
        const unsigned valid = rem >= 32 ? 0xFFFFFFFFu : ((1u << rem) - 1u);
        unsigned seen = *(volatile unsigned*)&mask[w];
        while (~seen & valid) {
            const int b = __ffs(~seen & valid) - 1;
            const unsigned prev = atomicOr(&mask[w], 1u << b);
            if (!(prev & (1u << b))) {
                __threadfence();    // the previous holder's writes precede ours
                return 32 * w + b;
            }
            seen |= prev | (1u << b);
        }
    }
    return -1;
}

// Persistent scoring kernel over one job: each block repeatedly takes the
// next hypothesis index from a device counter (zero at launch) and scores
// it.  The job is read from the kernel parameters, so its fields are
// constant-bank operands.  MODE kModeTree: the job's hypotheses are edges of the
// Monotone Scene Generation tree from the state in job.tree.  At most 64
// registers per thread (128 and 256 threads): four 256-thread blocks, 32 warps,
// fit an SM when the block's shared memory allows (the default launch shape),
// which hides latency better than three blocks of 80 registers.
template <int NT, int MODE, bool BINS>
__global__ void __launch_bounds__(NT, NT == 512 ? 1 : 1024 / NT) k_score(ScoreArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float s_pose[12];
    __shared__ int s_rbox[4], s_vbox[4], s_k32, s_next, s_slot, s_refused, s_bin_cnt[kBinTiles], s_jo_next,
        s_raster_done, s_vbounds[4];
    __shared__ long long s_h;
    __shared__ int s_red[3][NT / 32];

    SmemLayout L = smem_layout(a.zcap_words, a.mark_words, NT);
    ScoreSmem S;
    S.zbuf = reinterpret_cast<uint32_t*>(smem);
    S.marks = reinterpret_cast<uint32_t*>(smem + L.marks);
    S.kept = reinterpret_cast<KeptPoint*>(smem + L.kept);
    S.probe = reinterpret_cast<WarpProbe*>(smem + L.probe);
    S.stage = reinterpret_cast<TriStage*>(smem + L.probe);
    S.next_batch = &s_next;
    S.refused = &s_refused;
    S.bin_cnt = s_bin_cnt;
    S.jo_next = &s_jo_next;
    S.raster_done = &s_raster_done;
    S.vbounds = s_vbounds;
    if (threadIdx.x == 0) s_slot = a.vcache ? claim_vslot(a.vmask, a.vslots) : -1;
    __syncthreads();
    unsigned long long* vc = s_slot >= 0 ? a.vcache + (size_t)s_slot * a.vstride : nullptr;
    for (;;) {
        if (threadIdx.x == 0) s_h = (long long)atomicAdd(a.next, 1u);
        __syncthreads();
        const long long h = s_h;
        if (h >= a.n) break;
        score_one<NT, MODE, BINS>(a, a.job, h, S, s_pose, s_rbox, s_vbox, &s_k32, s_red, vc);
    }
    // every thread has passed the barrier after its last use of the slot
    if (threadIdx.x == 0 && s_slot >= 0) {
        __threadfence();
        atomicAnd(&a.vmask[s_slot >> 5], ~(1u << (s_slot & 31)));
    }
}

size_t score_smem_bytes(const ScoreConfig& cfg, int mark_words)
{
    return smem_layout(cfg.zcap_words, mark_words, cfg.threads).total;
}

template <int NT, int MODE, bool BINS>
static int score_grid_nt(size_t smem)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(k_score<NT, MODE, BINS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_score<NT, MODE, BINS>, NT, smem) != cudaSuccess)
        return -1;
    return max(1, per) * max(1, sms);
}

template <int NT>
static int score_grid_all(size_t smem)
{
    // the specialisations share the vertex-cache pool: size for the smallest
    return min(min(score_grid_nt<NT, kModePlain, false>(smem), score_grid_nt<NT, kModePlain, true>(smem)),
               min(score_grid_nt<NT, kModeTree, false>(smem), score_grid_nt<NT, kModeEq3, false>(smem)));
}

int score_grid(const ScoreConfig& cfg, int mark_words)
{
    size_t smem = score_smem_bytes(cfg, mark_words);
    switch (cfg.threads) {
    case 128: return score_grid_all<128>(smem);
    case 512: return score_grid_all<512>(smem);
    default: return score_grid_all<256>(smem);
    }
}

// The kernel specialisation a launch runs on (tile bins: plain scoring only;
// the other modes rasterise every tile from the whole mesh).
template <int NT>
static const void* score_kernel(const ScoreArgs& a)
{
    if (a.job.tree.depth) return (const void*)k_score<NT, kModeTree, false>;
    if (a.job.sc.jo_mode == 1) return (const void*)k_score<NT, kModeEq3, false>;
    if (a.bin_cap > 0) return (const void*)k_score<NT, kModePlain, true>;
    return (const void*)k_score<NT, kModePlain, false>;
}

template <int NT>
static cudaError_t launch_score_nt(const ScoreArgs& a, const ScoreConfig& cfg, int grid, cudaStream_t s)
{
    const size_t smem = score_smem_bytes(cfg, a.mark_words);
    const unsigned g = (unsigned)(a.n < grid ? a.n : grid);
    const void* fn = score_kernel<NT>(a);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ScoreArgs copy = a;
    void* args[] = {&copy};
    return cudaLaunchKernel(fn, dim3(g), dim3(NT), args, smem, s);
}

template <int NT>
static cudaError_t add_score_node_nt(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                                     const ScoreArgs& a, const ScoreConfig& cfg, int grid,
                                     cudaGraphNode_t* out)
{
    const size_t smem = score_smem_bytes(cfg, a.mark_words);
    const void* fn = score_kernel<NT>(a);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ScoreArgs copy = a;
    void* args[] = {&copy};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(fn);
    kp.gridDim = dim3((unsigned)(a.n < grid ? a.n : grid));
    kp.blockDim = dim3(NT);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, g, deps, ndeps, &kp);
}

cudaError_t add_score_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                           const ScoreArgs& a, const ScoreConfig& cfg, int grid, cudaGraphNode_t* out)
{
    if (a.n <= 0 || a.n > 0xFFFFFFF0ll || grid <= 0 || a.job.tree.depth) return cudaErrorInvalidValue;
    switch (cfg.threads) {
    case 128: return add_score_node_nt<128>(g, deps, ndeps, a, cfg, grid, out);
    case 512: return add_score_node_nt<512>(g, deps, ndeps, a, cfg, grid, out);
    default: return add_score_node_nt<256>(g, deps, ndeps, a, cfg, grid, out);
    }
}

cudaError_t launch_score(const ScoreArgs& a, const ScoreConfig& cfg, int grid, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    if (grid <= 0) return cudaErrorInvalidValue;
    if (a.n > 0xFFFFFFF0ll) return cudaErrorInvalidValue;   // the counter is 32-bit
    switch (cfg.threads) {
    case 128: return launch_score_nt<128>(a, cfg, grid, s);
    case 512: return launch_score_nt<512>(a, cfg, grid, s);
    default: return launch_score_nt<256>(a, cfg, grid, s);
    }
}

// ---------------------------------------------------------------------------
// M2M GICP refinement (Sec. IV-A "Parallel M2M GICP")
// ---------------------------------------------------------------------------
//
// Per hypothesis (one block): render the mesh at the input pose, keep the
// visible, unoccluded pixels on the stride lattice as the source cloud (each
// with the camera-frame normal of its triangle), then iterate Gauss-Newton
// steps of the GICP objective against the observed cloud: every source point
// moved by the current increment is matched to its nearest observed point
// within delta (the radius search of the scorer), contributes 28 binary32
// terms (the 6x6 normal matrix's upper triangle, the gradient and r^T M r)
// that are rounded to multiples of 2^-24 and summed exactly in int64, and
// thread 0 solves the system in binary64 and updates the increment.  The
// fixed-point sums make the result independent of the summation order.

constexpr int kGicpTerms = 28;
constexpr int kGicpThreads = 128;   // four blocks per SM: source clouds are small
constexpr float kGicpScale = 16777216.0f;    // 2^24
constexpr float kGicpLimit = 1048576.0f;     // a correspondence with a larger |term| is skipped

__device__ __forceinline__ float3 cross_rn(float3 a, float3 b)
{
    return make_float3(__fsub_rn(__fmul_rn(a.y, b.z), __fmul_rn(a.z, b.y)),
                       __fsub_rn(__fmul_rn(a.z, b.x), __fmul_rn(a.x, b.z)),
                       __fsub_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
}

__device__ __forceinline__ float3 unit_or_zero(float3 c)
{
    const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(c.x, c.x), __fmul_rn(c.y, c.y)), __fmul_rn(c.z, c.z));
    if (!(len2 > 0.0f)) return make_float3(0.0f, 0.0f, 0.0f);
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(len2));
    return make_float3(__fmul_rn(c.x, inv), __fmul_rn(c.y, inv), __fmul_rn(c.z, inv));
}

__device__ __forceinline__ float3 sub_rn(float4 a, float4 b)
{
    return make_float3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}

// Object-frame unit normal of triangle t, vertex order as stored.
__device__ __forceinline__ float3 triangle_normal(const DevMesh& m, int t)
{
    const int4 tv = __ldg(&m.tris[t]);
    const float4 a = __ldg(&m.verts[tv.x]), b = __ldg(&m.verts[tv.y]), c = __ldg(&m.verts[tv.z]);
    return unit_or_zero(cross_rn(sub_rn(b, a), sub_rn(c, a)));
}

// R v for the 3x3 rotation stored row-major with row pitch `pitch`.
__device__ __forceinline__ float3 rotate_rn(const float* R, int pitch, float x, float y, float z)
{
    return make_float3(
        __fadd_rn(__fadd_rn(__fmul_rn(R[0], x), __fmul_rn(R[1], y)), __fmul_rn(R[2], z)),
        __fadd_rn(__fadd_rn(__fmul_rn(R[pitch], x), __fmul_rn(R[pitch + 1], y)), __fmul_rn(R[pitch + 2], z)),
        __fadd_rn(__fadd_rn(__fmul_rn(R[2 * pitch], x), __fmul_rn(R[2 * pitch + 1], y)),
                  __fmul_rn(R[2 * pitch + 2], z)));
}

__global__ void k_obs_normals(DevScene sc, int jump, float4* nrm)
{
    const int n = sc.W * sc.H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int u = i % sc.W, v = i / sc.W;
        float3 nv = make_float3(0.0f, 0.0f, 0.0f);
        const int dc = sc.depth[i];
        if (dc != 0 && u >= 1 && v >= 1 && u + 1 < sc.W && v + 1 < sc.H) {
            const int nu[4] = {u - 1, u + 1, u, u}, nvv[4] = {v, v, v - 1, v + 1};
            float3 P[4];
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int d = sc.depth[nvv[k] * sc.W + nu[k]];
                if (d == 0 || abs(d - dc) > jump) ok = false;
                else P[k] = back_project(sc, nu[k], nvv[k], (unsigned)d);
            }
            if (ok) {
                const float3 a = make_float3(__fsub_rn(P[1].x, P[0].x), __fsub_rn(P[1].y, P[0].y),
                                             __fsub_rn(P[1].z, P[0].z));
                const float3 b = make_float3(__fsub_rn(P[3].x, P[2].x), __fsub_rn(P[3].y, P[2].y),
                                             __fsub_rn(P[3].z, P[2].z));
                nv = unit_or_zero(cross_rn(a, b));
            }
        }
        nrm[i] = make_float4(nv.x, nv.y, nv.z, 0.0f);
    }
}

cudaError_t launch_obs_normals(const DevScene& sc, int normal_jump, float4* nrm, cudaStream_t s)
{
    const int n = sc.W * sc.H;
    if (n <= 0) return cudaSuccess;
    k_obs_normals<<<(n + 255) / 256, 256, 0, s>>>(sc, normal_jump, nrm);
    return cudaGetLastError();
}

// The 28 terms of one correspondence: p = Rf a + tf (already moved), m = Rf na,
// observed b with normal nb.  False (no terms) when the combined covariance is
// not positive or a term is out of bounds.
__device__ __forceinline__ bool gicp_terms(const float* Rf, float3 p, float4 na, float3 b, float4 nb,
                                           float eps, float* out)
{
    const float3 m = rotate_rn(Rf, 3, na.x, na.y, na.z);
    const float e = __fsub_rn(1.0f, eps);
    // C = 2 I - e (nb nb^T + m m^T)
    const float c00 = __fsub_rn(2.0f, __fmul_rn(e, __fadd_rn(__fmul_rn(nb.x, nb.x), __fmul_rn(m.x, m.x))));
    const float c11 = __fsub_rn(2.0f, __fmul_rn(e, __fadd_rn(__fmul_rn(nb.y, nb.y), __fmul_rn(m.y, m.y))));
    const float c22 = __fsub_rn(2.0f, __fmul_rn(e, __fadd_rn(__fmul_rn(nb.z, nb.z), __fmul_rn(m.z, m.z))));
    const float c01 = -__fmul_rn(e, __fadd_rn(__fmul_rn(nb.x, nb.y), __fmul_rn(m.x, m.y)));
    const float c02 = -__fmul_rn(e, __fadd_rn(__fmul_rn(nb.x, nb.z), __fmul_rn(m.x, m.z)));
    const float c12 = -__fmul_rn(e, __fadd_rn(__fmul_rn(nb.y, nb.z), __fmul_rn(m.y, m.z)));
    // M = C^-1 (adjugate over determinant)
    const float a00 = __fsub_rn(__fmul_rn(c11, c22), __fmul_rn(c12, c12));
    const float a01 = __fsub_rn(__fmul_rn(c02, c12), __fmul_rn(c01, c22));
    const float a02 = __fsub_rn(__fmul_rn(c01, c12), __fmul_rn(c02, c11));
    const float a11 = __fsub_rn(__fmul_rn(c00, c22), __fmul_rn(c02, c02));
    const float a12 = __fsub_rn(__fmul_rn(c01, c02), __fmul_rn(c00, c12));
    const float a22 = __fsub_rn(__fmul_rn(c00, c11), __fmul_rn(c01, c01));
    const float det = __fadd_rn(__fadd_rn(__fmul_rn(c00, a00), __fmul_rn(c01, a01)), __fmul_rn(c02, a02));
    if (!(det > 0.0f)) return false;
    const float id = __fdiv_rn(1.0f, det);
    float M[3][3];
    M[0][0] = __fmul_rn(a00, id); M[0][1] = __fmul_rn(a01, id); M[0][2] = __fmul_rn(a02, id);
    M[1][1] = __fmul_rn(a11, id); M[1][2] = __fmul_rn(a12, id); M[2][2] = __fmul_rn(a22, id);
    M[1][0] = M[0][1]; M[2][0] = M[0][2]; M[2][1] = M[1][2];
    const float r[3] = {__fsub_rn(b.x, p.x), __fsub_rn(b.y, p.y), __fsub_rn(b.z, p.z)};
    // Jacobian of r with respect to (w, v) is [ [p]x , -I ]; MA = M [p]x
    float MA[3][3], AMA[3][3], Mr[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        MA[i][0] = __fsub_rn(__fmul_rn(M[i][1], p.z), __fmul_rn(M[i][2], p.y));
        MA[i][1] = __fsub_rn(__fmul_rn(M[i][2], p.x), __fmul_rn(M[i][0], p.z));
        MA[i][2] = __fsub_rn(__fmul_rn(M[i][0], p.y), __fmul_rn(M[i][1], p.x));
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        AMA[0][j] = __fsub_rn(__fmul_rn(p.z, MA[1][j]), __fmul_rn(p.y, MA[2][j]));
        AMA[1][j] = __fsub_rn(__fmul_rn(p.x, MA[2][j]), __fmul_rn(p.z, MA[0][j]));
        AMA[2][j] = __fsub_rn(__fmul_rn(p.y, MA[0][j]), __fmul_rn(p.x, MA[1][j]));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
        Mr[i] = __fadd_rn(__fadd_rn(__fmul_rn(M[i][0], r[0]), __fmul_rn(M[i][1], r[1])), __fmul_rn(M[i][2], r[2]));
    int k = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = i; j < 6; ++j) {
            float h;
            if (i < 3 && j < 3) h = AMA[i][j];
            else if (i < 3) h = -MA[j - 3][i];
            else h = M[i - 3][j - 3];
            out[k++] = h;
        }
    }
    out[k++] = __fsub_rn(__fmul_rn(p.z, Mr[1]), __fmul_rn(p.y, Mr[2]));
    out[k++] = __fsub_rn(__fmul_rn(p.x, Mr[2]), __fmul_rn(p.z, Mr[0]));
    out[k++] = __fsub_rn(__fmul_rn(p.y, Mr[0]), __fmul_rn(p.x, Mr[1]));
    out[k++] = -Mr[0];
    out[k++] = -Mr[1];
    out[k++] = -Mr[2];
    out[k++] = __fadd_rn(__fadd_rn(__fmul_rn(r[0], Mr[0]), __fmul_rn(r[1], Mr[1])), __fmul_rn(r[2], Mr[2]));
    bool ok = true;
#pragma unroll
    for (int i = 0; i < kGicpTerms; ++i) ok = ok && fabsf(out[i]) < kGicpLimit;
    return ok;
}

// rint(v) as a 64-bit integer for |v| < 2^46 without a 64-bit conversion:
// below 2^31 a 32-bit round to nearest even; above, v is already an integer
// (its ulp is at least 2^8) and splits exactly as 2^16 h + l, h = trunc(v /
// 2^16) (the scaling is exact) and l = v - 2^16 h (exact: a multiple of 2^8
// below 2^16 in magnitude).
__device__ __forceinline__ long long rint_to_ll(float v)
{
    if (fabsf(v) < 2147483648.0f) return (long long)__float2int_rn(v);
    const float h = truncf(__fmul_rn(v, 1.0f / 65536.0f));
    const float l = __fsub_rn(v, __fmul_rn(h, 65536.0f));
    return (long long)__float2int_rz(h) * 65536ll + (long long)__float2int_rz(l);
}

// H xi = -g from the fixed-point sums, by Cholesky in binary64 (one thread).
__device__ bool gicp_solve(const unsigned long long* S, double* xi)
{
    double H[6][6], g[6], L[6][6], y[6];
    int k = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) {
            H[i][j] = __ddiv_rn(__ll2double_rn((long long)S[k++]), 16777216.0);
            H[j][i] = H[i][j];
        }
    for (int i = 0; i < 6; ++i) g[i] = __ddiv_rn(__ll2double_rn((long long)S[k++]), 16777216.0);
    for (int j = 0; j < 6; ++j) {
        double s = H[j][j];
        for (int q = 0; q < j; ++q) s = __dsub_rn(s, __dmul_rn(L[j][q], L[j][q]));
        if (!(s > 0.0)) return false;
        L[j][j] = __dsqrt_rn(s);
        for (int i = j + 1; i < 6; ++i) {
            double t = H[i][j];
            for (int q = 0; q < j; ++q) t = __dsub_rn(t, __dmul_rn(L[i][q], L[j][q]));
            L[i][j] = __ddiv_rn(t, L[j][j]);
        }
    }
    for (int i = 0; i < 6; ++i) {
        double t = -g[i];
        for (int q = 0; q < i; ++q) t = __dsub_rn(t, __dmul_rn(L[i][q], y[q]));
        y[i] = __ddiv_rn(t, L[i][i]);
    }
    for (int i = 5; i >= 0; --i) {
        double t = y[i];
        for (int q = i + 1; q < 6; ++q) t = __dsub_rn(t, __dmul_rn(L[q][i], xi[q]));
        xi[i] = __ddiv_rn(t, L[i][i]);
    }
    return true;
}

// Apply the step xi to the increment (R, t): R <- dR R, t <- dR t + v, with
// dR the rotation of the quaternion (1, w/2) normalised.  True when the step
// is below the stopping thresholds.
__device__ bool gicp_update(double* R, double* t, const double* xi, float stop_rot, float stop_trans)
{
    const double hx = __dmul_rn(xi[0], 0.5), hy = __dmul_rn(xi[1], 0.5), hz = __dmul_rn(xi[2], 0.5);
    const double nrm = __dsqrt_rn(__dadd_rn(__dadd_rn(__dadd_rn(1.0, __dmul_rn(hx, hx)), __dmul_rn(hy, hy)),
                                            __dmul_rn(hz, hz)));
    const double qw = __ddiv_rn(1.0, nrm), qx = __ddiv_rn(hx, nrm), qy = __ddiv_rn(hy, nrm), qz = __ddiv_rn(hz, nrm);
    double d[9];
    d[0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(qy, qy), __dmul_rn(qz, qz))));
    d[1] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(qx, qy), __dmul_rn(qw, qz)));
    d[2] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(qx, qz), __dmul_rn(qw, qy)));
    d[3] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(qx, qy), __dmul_rn(qw, qz)));
    d[4] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qz, qz))));
    d[5] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(qy, qz), __dmul_rn(qw, qx)));
    d[6] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(qx, qz), __dmul_rn(qw, qy)));
    d[7] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(qy, qz), __dmul_rn(qw, qx)));
    d[8] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy))));
    double R2[9], t2[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            R2[3 * i + j] = __dadd_rn(__dadd_rn(__dmul_rn(d[3 * i], R[j]), __dmul_rn(d[3 * i + 1], R[3 + j])),
                                      __dmul_rn(d[3 * i + 2], R[6 + j]));
        t2[i] = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(d[3 * i], t[0]), __dmul_rn(d[3 * i + 1], t[1])),
                                    __dmul_rn(d[3 * i + 2], t[2])), xi[3 + i]);
    }
    for (int i = 0; i < 9; ++i) R[i] = R2[i];
    for (int i = 0; i < 3; ++i) t[i] = t2[i];
    const double sr = (double)stop_rot, st = (double)stop_trans;
    const double w2 = __dadd_rn(__dadd_rn(__dmul_rn(xi[0], xi[0]), __dmul_rn(xi[1], xi[1])), __dmul_rn(xi[2], xi[2]));
    const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(xi[3], xi[3]), __dmul_rn(xi[4], xi[4])), __dmul_rn(xi[5], xi[5]));
    return w2 < __dmul_rn(sr, sr) && v2 < __dmul_rn(st, st);
}

// Render the hypothesis in z-buffer tiles and append its source cloud
// (visible, unoccluded pixels on the stride lattice) to src; *count ends as
// the number of source points (entries past cap are not written).
template <int NT, bool K32, bool VC>
__device__ void gicp_source(const GicpArgs& a, const Job& J, const float* P, const unsigned long long* vc,
                            const int* rbox, uint32_t* zbuf, char* probe, float4* src, int* count)
{
    const DevScene& sc = J.sc;
    const int warp = threadIdx.x >> 5;
    TriStage* TS = reinterpret_cast<TriStage*>(probe + warp * kWarpScratch);
    const int s = sc.stride;
    const int rw = rbox[2] - rbox[0], rh = rbox[3] - rbox[1];
    if (rw <= 0 || rh <= 0) return;
    const int cap_px = K32 ? a.zcap_words : a.zcap_words / 2;
    const int tw = min(rw, cap_px);
    const int th = max(1, cap_px / tw);
    for (int tv0 = rbox[1]; tv0 < rbox[3]; tv0 += th) {
        for (int tu0 = rbox[0]; tu0 < rbox[2]; tu0 += tw) {
            const int tu1 = min(tu0 + tw, rbox[2]), tv1 = min(tv0 + th, rbox[3]);
            const int words = K32 ? tw * (tv1 - tv0) : 2 * tw * (tv1 - tv0);
            for (int i = threadIdx.x; i < words; i += NT) zbuf[i] = 0xFFFFFFFFu;
            __syncthreads();
            raster_tile<NT, K32, VC>(sc, J.m, P, vc, TS, zbuf, tu0, tv0, tu1, tv1, tw, a.err);
            __syncthreads();
            const int us0 = ((tu0 + s - 1) / s) * s, vs0 = ((tv0 + s - 1) / s) * s;
            const int nu = us0 < tu1 ? (tu1 - 1 - us0) / s + 1 : 0;
            const int nv = vs0 < tv1 ? (tv1 - 1 - vs0) / s + 1 : 0;
            for (int k = threadIdx.x; k < nu * nv; k += NT) {
                const int kv = div_small(k, nu);
                const int u = us0 + (k - kv * nu) * s, v = vs0 + kv * s;
                const int zi = (v - tv0) * tw + (u - tu0);
                unsigned d = 0;
                int tri = -1;
                if (K32) {
                    const uint32_t w = zbuf[zi];
                    if (w != 0xFFFFFFFFu) { d = w >> 16; tri = (int)(w & 0xFFFFu); }
                } else {
                    const unsigned long long w = reinterpret_cast<unsigned long long*>(zbuf)[zi];
                    if (w != kEmptyKey) { d = (unsigned)(w >> 32); tri = (int)(uint32_t)w; }
                }
                if (tri < 0) continue;
                const int pix = v * sc.W + u;
                const unsigned dobs = __ldg(&sc.depth[pix]);
                const bool occluded = sc.occ_margin >= 0 && dobs > 0 &&
                                      (unsigned long long)dobs + (unsigned)sc.occ_margin < d &&
                                      (J.label < 0 || __ldg(&sc.labels[pix]) != J.label);
                if (occluded) continue;
                const float3 q = back_project(sc, u, v, d);
                const float3 no = triangle_normal(J.m, tri);
                const float3 nc = rotate_rn(P, 4, no.x, no.y, no.z);
                const int idx = atomicAdd(count, 1);
                if (idx < a.src_cap) {
                    src[2 * (size_t)idx] = make_float4(q.x, q.y, q.z, 0.0f);
                    src[2 * (size_t)idx + 1] = make_float4(nc.x, nc.y, nc.z, 0.0f);
                }
            }
            __syncthreads();
        }
    }
}

__host__ __device__ inline size_t gicp_probe_offset(int zcap_words)
{
    return align16(sizeof(uint32_t) * (size_t)zcap_words);
}

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_gicp(GicpArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float s_pose[12], s_Rf[9], s_tf[3];
    __shared__ double s_R[9], s_t[3];
    __shared__ unsigned long long s_sum[kGicpTerms];
    __shared__ int s_rbox[4], s_k32, s_slot, s_nsrc, s_corr, s_done, s_updates, s_last;
    __shared__ long long s_h;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Job& J = a.job;
    const DevScene& sc = J.sc;
    uint32_t* zbuf = reinterpret_cast<uint32_t*>(smem);
    char* probe = reinterpret_cast<char*>(smem) + gicp_probe_offset(a.zcap_words);
    WarpProbe& WP = *reinterpret_cast<WarpProbe*>(probe + warp * kWarpScratch);
    if (threadIdx.x == 0) {
        s_slot = claim_vslot(a.smask, a.slots);
        if (s_slot < 0) atomicOr(a.err, kErrNoSlot);
    }
    __syncthreads();
    if (s_slot < 0) return;
    const unsigned long long* vc = a.vcache ? a.vcache + (size_t)s_slot * a.vstride : nullptr;
    float4* src = a.src + (size_t)s_slot * 2 * (size_t)a.src_cap;
    const MarkBand nomark = {nullptr, 0, 0, 0, 0, 0, a.err};
    for (;;) {
        if (threadIdx.x == 0) s_h = (long long)atomicAdd(a.next, 1u);
        __syncthreads();
        const long long h = s_h;
        if (h >= a.n) break;
        if (threadIdx.x < 12) s_pose[threadIdx.x] = J.poses[h * 12 + threadIdx.x];
        if (threadIdx.x == 0) s_nsrc = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            float zmax;
            project_box(sc, s_pose, J.m.lo, J.m.hi, J.roi[0], J.roi[1], J.roi[2], J.roi[3], s_rbox, &zmax);
            s_k32 = (J.m.n_tris <= 65535 && zmax < 6.5f) ? 1 : 0;
        }
        if (vc) vertex_pass(sc, J.m, s_pose, const_cast<unsigned long long*>(vc), NT);
        __syncthreads();
        if (s_k32) {
            if (vc) gicp_source<NT, true, true>(a, J, s_pose, vc, s_rbox, zbuf, probe, src, &s_nsrc);
            else gicp_source<NT, true, false>(a, J, s_pose, vc, s_rbox, zbuf, probe, src, &s_nsrc);
        } else {
            if (vc) gicp_source<NT, false, true>(a, J, s_pose, vc, s_rbox, zbuf, probe, src, &s_nsrc);
            else gicp_source<NT, false, false>(a, J, s_pose, vc, s_rbox, zbuf, probe, src, &s_nsrc);
        }
        const int nsrc = s_nsrc;
        if (nsrc > a.src_cap) {
            // the source cloud does not fit its slot: the pose is returned unchanged
            if (threadIdx.x < 12) a.poses_out[h * 12 + threadIdx.x] = s_pose[threadIdx.x];
            if (threadIdx.x == 0) {
                atomicOr(a.err, kErrSourceCap);
                if (a.info) { a.info[2 * h] = -1; a.info[2 * h + 1] = nsrc; }
            }
            __syncthreads();
            continue;
        }
        if (threadIdx.x == 0) {
            for (int i = 0; i < 9; ++i) { s_R[i] = (i % 4 == 0) ? 1.0 : 0.0; s_Rf[i] = (float)s_R[i]; }
            for (int i = 0; i < 3; ++i) { s_t[i] = 0.0; s_tf[i] = 0.0f; }
            s_done = 0;
            s_updates = 0;
            s_last = 0;
        }
        __syncthreads();
        for (int it = 0; it < a.max_iters; ++it) {
            if (threadIdx.x < kGicpTerms) s_sum[threadIdx.x] = 0ull;
            if (threadIdx.x == 0) s_corr = 0;
            __syncthreads();
            long long acc = 0;
            int corr = 0;
            for (int base = warp * 32; base < nsrc; base += NT) {
                const int i = base + lane;
                const bool valid = i < nsrc;
                float4 A = make_float4(0.f, 0.f, 0.f, 0.f), NA = A;
                if (valid) { A = src[2 * (size_t)i]; NA = src[2 * (size_t)i + 1]; }
                const float3 r0 = rotate_rn(s_Rf, 3, A.x, A.y, A.z);
                const float3 p = make_float3(__fadd_rn(r0.x, s_tf[0]), __fadd_rn(r0.y, s_tf[1]),
                                             __fadd_rn(r0.z, s_tf[2]));
                const unsigned long long nn = probe_batch<false>(sc, valid, p.x, p.y, p.z, 0u, WP, lane, nomark);
                bool ok = valid && nn != kEmptyKey;
                float terms[kGicpTerms];
                if (ok) {
                    const uint32_t pw = (uint32_t)nn;
                    const int pu = (int)(pw & 0xFFFFu), pv = (int)(pw >> 16);
                    const int pix = pv * sc.W + pu;
                    const float3 b = back_project(sc, pu, pv, __ldg(&sc.depth[pix]));
                    ok = gicp_terms(s_Rf, p, NA, b, __ldg(&a.nrm[pix]), a.epsilon, terms);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                corr += __popc(bal);
                if (bal) {
#pragma unroll
                    for (int j = 0; j < kGicpTerms; ++j) {
                        long long q = ok ? rint_to_ll(__fmul_rn(terms[j], kGicpScale)) : 0ll;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
                        if (lane == j) acc += q;
                    }
                }
            }
            if (lane < kGicpTerms) atomicAdd(&s_sum[lane], (unsigned long long)acc);
            if (lane == 0) atomicAdd(&s_corr, corr);
            __syncthreads();
            if (threadIdx.x == 0) {
                s_last = s_corr;
                double xi[6];
                if (s_corr < a.min_corr || !gicp_solve(s_sum, xi)) {
                    s_done = 1;
                } else {
                    if (gicp_update(s_R, s_t, xi, a.stop_rot, a.stop_trans)) s_done = 1;
                    ++s_updates;
                    for (int i = 0; i < 9; ++i) s_Rf[i] = __double2float_rn(s_R[i]);
                    for (int i = 0; i < 3; ++i) s_tf[i] = __double2float_rn(s_t[i]);
                }
            }
            __syncthreads();
            if (s_done) break;
        }
        // refined pose = increment o input pose
        if (threadIdx.x < 12) {
            const int i = threadIdx.x / 4, j = threadIdx.x % 4;
            const float* P = s_pose;
            double x;
            if (j < 3) {
                x = __dadd_rn(__dadd_rn(__dmul_rn(s_R[3 * i], (double)P[j]), __dmul_rn(s_R[3 * i + 1], (double)P[4 + j])),
                              __dmul_rn(s_R[3 * i + 2], (double)P[8 + j]));
            } else {
                x = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(s_R[3 * i], (double)P[3]),
                                                  __dmul_rn(s_R[3 * i + 1], (double)P[7])),
                                        __dmul_rn(s_R[3 * i + 2], (double)P[11])), s_t[i]);
            }
            a.poses_out[h * 12 + threadIdx.x] = __double2float_rn(x);
        }
        if (threadIdx.x == 0 && a.info) {
            a.info[2 * h] = s_updates;
            a.info[2 * h + 1] = s_last;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAnd(&a.smask[s_slot >> 5], ~(1u << (s_slot & 31)));
    }
}

size_t gicp_smem_bytes(int zcap_words)
{
    return gicp_probe_offset(zcap_words) + kWarpScratch * (kGicpThreads / 32);
}

int gicp_grid(int zcap_words)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = gicp_smem_bytes(zcap_words);
    if (cudaFuncSetAttribute(k_gicp<kGicpThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gicp<kGicpThreads>, kGicpThreads, smem) != cudaSuccess)
        return -1;
    return max(1, per) * max(1, sms);
}

cudaError_t launch_gicp(const GicpArgs& a, int grid, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    if (a.n > 0xFFFFFFF0ll || grid <= 0 || grid > a.slots) return cudaErrorInvalidValue;
    const size_t smem = gicp_smem_bytes(a.zcap_words);
    cudaError_t e = cudaFuncSetAttribute(k_gicp<kGicpThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gicp<kGicpThreads><<<(unsigned)(a.n < grid ? a.n : grid), kGicpThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 6-DoF pose proposals (Sec. V-B, Eq. 5 and Eq. 6)
// ---------------------------------------------------------------------------

__global__ void k_mask_depth_range(ProposalArgs a)
{
    const int bw = a.box[2] - a.box[0], bh = a.box[3] - a.box[1];
    unsigned lo = 0xFFFFFFFFu, hi = 0u;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bw * bh; i += gridDim.x * blockDim.x) {
        const int u = a.box[0] + i % bw, v = a.box[1] + i / bw;
        const int pix = v * a.sc.W + u;
        const unsigned d = a.sc.depth[pix];
        if (d != 0 && a.sc.labels[pix] == a.label) {
            lo = min(lo, d);
            hi = max(hi, d);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0 && hi != 0u) {
        atomicMin(&a.zr[0], lo);
        atomicMax(&a.zr[1], hi);
    }
}

__global__ void k_proposals(ProposalArgs a)
{
    const long long total = (long long)a.M * a.N * a.K;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx == 0 && a.z_out) {
        const bool any = a.zr[1] != 0u;
        a.z_out[0] = any ? (int32_t)a.zr[0] : 0;
        a.z_out[1] = any ? (int32_t)a.zr[1] : 0;
    }
    if (idx >= total) return;
    const int j = (int)(idx % a.K);
    const int k = (int)((idx / a.K) % a.N);
    const int i = (int)(idx / ((long long)a.K * a.N));
    // viewpoint i of the Fibonacci lattice (object frame, towards the camera)
    const float golden = 2.39996322972865332f;          // pi (3 - sqrt 5)
    const float y = 1.0f - (2.0f * i + 1.0f) / (float)a.M;
    const float rad = sqrtf(fmaxf(0.0f, 1.0f - y * y));
    const float phi = golden * (float)i;
    const float vx = rad * cosf(phi), vy = y, vz = rad * sinf(phi);
    // camera axes in the object frame: forward = -v, right, down
    const float fx = -vx, fy = -vy, fz = -vz;
    float rx = fy * 1.0f - fz * 0.0f, ry = fz * 0.0f - fx * 1.0f, rz = 0.0f;   // forward x (0,0,1)
    float rn = sqrtf(rx * rx + ry * ry + rz * rz);
    if (rn < 1e-6f) {                                   // forward parallel to z: use (0,1,0)
        rx = fy * 0.0f - fz * 1.0f;
        ry = fz * 0.0f - fx * 0.0f;
        rz = fx * 1.0f - fy * 0.0f;
        rn = sqrtf(rx * rx + ry * ry + rz * rz);
    }
    rx /= rn; ry /= rn; rz /= rn;
    const float dx = fy * rz - fz * ry, dy = fz * rx - fx * rz, dz = fx * ry - fy * rx;
    // in-plane rotation about the optical axis
    const float th = 6.28318530717958648f * (float)k / (float)a.N;
    const float c = cosf(th), s = sinf(th);
    const float R[9] = {c * rx - s * dx, c * ry - s * dy, c * rz - s * dz,
                        s * rx + c * dx, s * ry + c * dy, s * rz + c * dz,
                        fx, fy, fz};
    // translation: the box centre back-projected at depth z_j
    const bool any = a.zr[1] != 0u;
    const float zmin = any ? (float)a.zr[0] / 10000.0f : 0.0f;
    const float zmax = any ? (float)a.zr[1] / 10000.0f : 0.0f;
    const float z = a.K > 1 ? zmin + (zmax - zmin) * (float)j / (float)(a.K - 1) : 0.5f * (zmin + zmax);
    const float uc = 0.5f * (float)(a.box[0] + a.box[2] - 1), vc = 0.5f * (float)(a.box[1] + a.box[3] - 1);
    const float cxp = (uc - a.sc.cx) * z / a.sc.fx, cyp = (vc - a.sc.cy) * z / a.sc.fy;
    float* out = a.poses + 12 * idx;
    const float m0 = a.centre[0], m1 = a.centre[1], m2 = a.centre[2];
    out[0] = R[0]; out[1] = R[1]; out[2] = R[2];
    out[3] = cxp - (R[0] * m0 + R[1] * m1 + R[2] * m2);
    out[4] = R[3]; out[5] = R[4]; out[6] = R[5];
    out[7] = cyp - (R[3] * m0 + R[4] * m1 + R[5] * m2);
    out[8] = R[6]; out[9] = R[7]; out[10] = R[8];
    out[11] = z - (R[6] * m0 + R[7] * m1 + R[8] * m2);
}

cudaError_t launch_proposals(const ProposalArgs& a, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(a.zr, 0xFF, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.zr + 1, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int area = (a.box[2] - a.box[0]) * (a.box[3] - a.box[1]);
    if (area > 0) k_mask_depth_range<<<min(1024, (area + 255) / 256), 256, 0, s>>>(a);
    const long long total = (long long)a.M * a.N * a.K;
    k_proposals<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// argmin of J = J_o + J_r (warp shuffles, then the last block reduces the partials)
// ---------------------------------------------------------------------------

constexpr int kBestThreads = 256;

struct BestKey {
    unsigned long long hi;   // (J << 32) | 0
    unsigned long long id;   // caller id or index
    long long idx;
};

__device__ __forceinline__ bool best_less(const BestKey& x, const BestKey& y)
{
    if (x.hi != y.hi) return x.hi < y.hi;
    if (x.id != y.id) return x.id < y.id;
    return x.idx < y.idx;
}

__device__ __forceinline__ BestKey shfl_best(const BestKey& k, int o)
{
    BestKey r;
    r.hi = __shfl_xor_sync(0xffffffffu, k.hi, o);
    r.id = __shfl_xor_sync(0xffffffffu, k.id, o);
    r.idx = __shfl_xor_sync(0xffffffffu, k.idx, o);
    return r;
}

__device__ BestKey block_best(BestKey k, BestKey* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        BestKey t = shfl_best(k, o);
        if (best_less(t, k)) k = t;
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = k;
    __syncthreads();
    if (w == 0) {
        BestKey none = {~0ull, ~0ull, 0x7FFFFFFFFFFFFFFFll};
        k = lane < kBestThreads / 32 ? sh[lane] : none;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            BestKey t = shfl_best(k, o);
            if (best_less(t, k)) k = t;
        }
    }
    return k;
}

__global__ void __launch_bounds__(kBestThreads) k_best(BestArgs a)
{
    __shared__ BestKey sh[kBestThreads / 32];
    __shared__ bool last;
    BestKey k = {~0ull, ~0ull, 0x7FFFFFFFFFFFFFFFll};
    for (long long i = blockIdx.x * (long long)kBestThreads + threadIdx.x; i < a.n;
         i += (long long)gridDim.x * kBestThreads) {
        long long J = (long long)a.costs[2 * i] + a.costs[2 * i + 1];
        BestKey c = {(unsigned long long)J << 32, a.ids ? a.ids[i] : (unsigned long long)i, i};
        if (best_less(c, k)) k = c;
    }
    k = block_best(k, sh);
    if (threadIdx.x == 0) {
        a.partial[3 * blockIdx.x + 0] = k.hi;
        a.partial[3 * blockIdx.x + 1] = k.id;
        a.partial[3 * blockIdx.x + 2] = (unsigned long long)k.idx;
        __threadfence();
        unsigned t = atomicAdd(a.ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    BestKey m = {~0ull, ~0ull, 0x7FFFFFFFFFFFFFFFll};
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kBestThreads) {
        BestKey c = {a.partial[3 * b], a.partial[3 * b + 1], (long long)a.partial[3 * b + 2]};
        if (best_less(c, m)) m = c;
    }
    __syncthreads();
    m = block_best(m, sh);
    if (threadIdx.x == 0) {
        if (a.best_index) *a.best_index = m.idx;
        if (a.best_cost) *a.best_cost = (int32_t)(m.hi >> 32);
        // (J << 32) | id: the smallest such key over several shards is their winner
        if (a.key) *a.key = m.hi | (m.id & 0xFFFFFFFFull);
        *a.ticket = 0u;
    }
}

int best_blocks(long long n)
{
    long long b = (n + kBestThreads - 1) / kBestThreads;
    return (int)(b < 1 ? 1 : (b > kBestMaxBlocks ? kBestMaxBlocks : b));
}

cudaError_t launch_best(const BestArgs& a, cudaStream_t s)
{
    k_best<<<best_blocks(a.n), kBestThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace perch
