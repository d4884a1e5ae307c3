// Internal types shared by the host API (perch_api.cu and its siblings) and the kernels
// (perch_kernels.cu) of libperch.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace perch {

constexpr uint64_t kEmptyKey = ~0ull;          // empty hash slot / empty z-buffer word
constexpr int kCellBias = 1 << 20;             // cell coordinates packed as 21-bit fields
constexpr float kCellGrow = 1.0f + 1.0f / 64.0f;  // hash cell edge = delta * kCellGrow
constexpr double kMaxCellCoord = 1.0e5;        // |coordinate / cell| bound for exact probing

// Device-resident observation (read-only during scoring).
struct DevScene {
    int W, H;
    float fx, fy, cx, cy;
    float delta, delta2, cell, inv_cell, tau_c, z_near;   // inv_cell = fl(1 / cell)
    int color_check, stride, occ_margin;
    int jo_mode;              // 0: NN marks (Sec. IV-A kernel); 1: Eq. 3 with the Eq. 2 test
    const uint16_t* depth;    // H*W
    const int32_t* labels;    // H*W or nullptr
    const float4* lab;        // H*W: (L, a, b, 0)
    const float4* pxyz;       // H*W: back-projected point of each pixel of I, w = 1 (w = 0: not in I)
    const float4* pts;        // n_pts, grouped by hash cell: (x, y, z, (v << 16 | u) bits)
    const uint4* table;       // hash slots: (key lo, key hi, start, count)
    uint32_t table_mask;
    int n_pts;
    // bit per hash cell in the box [near_lo, near_lo + near_n): set iff one of
    // the cell's 27 neighbours (itself included) holds an observed point;
    // cells outside the box have none.  nullptr: no filter.
    const uint32_t* near_bits;
    int near_lo[3], near_n[3];
    // dense cell index over the same box (z-major, then y, then x): pts is
    // sorted by cell and cell c holds pts[cell_start[c], cell_start[c + 1]),
    // so the three cells x-1..x+1 of a row are one contiguous run.  nullptr:
    // the box is too large, the hash table is used instead.
    const uint32_t* cell_start;
};

// Device-resident mesh.
struct DevMesh {
    const float4* verts;      // (x, y, z, rgb packed in the low 24 bits of w's bit pattern)
    const int4* tris;         // (a, b, c, 0)
    int n_verts, n_tris;
    float vol_r, vol_h;
    float lo[3], hi[3];       // object-frame bounding box of the vertices
};

// A state of the Monotone Scene Generation tree (the objects placed so
// far) as per-pixel images, for scoring the edges that add one more object.
struct TreeState {
    const uint32_t* depth;    // W*H composed depth of the placed objects (0 = none), or nullptr
    const uint32_t* mark;     // W*H bits: observed pixels explained by a placed object
    const uint32_t* vol;      // W*H bits: observed pixels already counted in J_o
    uint32_t* out_depth;      // child state (pre-copied from the parent), or nullptr
    uint32_t* out_mark;
    uint32_t* out_vol;
    int margin;               // occlusion margin (0.1 mm)
};

// One work item: n hypotheses of one mesh against one scene.
struct Job {
    DevScene sc;
    DevMesh m;
    int label;                // -1: cylinder V(O); >= 0: label V(O)
    int roi[4];               // clipped to the image, half-open
    const float* poses;       // n*12 (device)
    int32_t* costs;           // n*2 (device)
    long long n;
    TreeState tree;           // tree.depth == nullptr: plain scoring
};

// One scoring launch: the hypotheses of one job.  Launches that may run at
// the same time (the jobs of one batch) share the vertex-cache pool.
struct ScoreArgs {
    Job job;                  // read from the parameter bank
    long long n;              // hypotheses (= job.n)
    int zcap_words;           // z-buffer capacity in 32-bit words
    int mark_words;           // marks bitset capacity in 32-bit words
    unsigned long long* dump; // debug: W*H 64-bit keys, or nullptr
    int* err;                 // device error word (bit flags)
    unsigned* next;           // hypothesis counter, zeroed before the launch
    unsigned long long* vcache;  // vertex-cache pool: vslots slots of vstride vertices, or nullptr
    long long vstride;
    unsigned* vmask;          // (vslots + 31) / 32 words, bit set = slot in use; zero when idle
    int vslots;
    // z-buffer tile bins: when a hypothesis's pixel box needs 2 .. kBinTiles
    // tiles, each tile's triangles are listed first (bin_cap ids per tile, as
    // int32 at 8-byte offset bin_off of the block's vertex-cache slot) and the
    // tile rasterises only those; 0 = no bins.
    int bin_cap;
    long long bin_off;
};

// Most z-buffer tiles a hypothesis may be binned into.
constexpr int kBinTiles = 32;

// Error bits written by kernels into the context's error word.
enum : int { kErrKeyRange = 1, kErrMarkCap = 2, kErrHashFull = 4, kErrSourceCap = 8, kErrNoSlot = 16,
             kErrCheck = 32 };

// Debug builds (PERCH_CHECKS defined: build.py's checks=True, libperch_checks.so)
// test shared- and global-memory indexes of the scorer before each access:
// PERCH_CHECKED(cond, err) is false when cond fails, after setting kErrCheck
// in the error word (err may be null), so the caller skips the access and
// the host reports the violation.  Nothing traps.  In normal builds it is
// the constant true and costs nothing.
#ifdef PERCH_CHECKS
__device__ __forceinline__ bool perch_checked(bool ok, int* err)
{
    if (!ok && err) atomicOr(err, kErrCheck);
    return ok;
}
#define PERCH_CHECKED(cond, err) ::perch::perch_checked((cond), (err))
#else
#define PERCH_CHECKED(cond, err) true
#endif

// Launch configuration of the scoring kernel (chosen by the host; the
// autotuner searches over these).
struct ScoreConfig {
    int threads;              // 128, 256 or 512
    int zcap_words;           // z-buffer words (32-bit keys: pixels; 64-bit: half)
    int mark_bits;            // admissible-box bitset capacity in bits
    int bin_cap;              // triangles per z-buffer tile bin, 0 = no bins
};

// 8-byte words of one vertex-cache slot: the vertex records, then (bin_cap > 0)
// kBinTiles bins of bin_cap int32 triangle ids.
inline long long vcache_slot_words(int max_verts, int bin_cap, long long* bin_off)
{
    const long long v = ((long long)max_verts + 31) / 32 * 32;
    *bin_off = v;
    return bin_cap > 0 ? v + ((long long)kBinTiles * bin_cap + 63) / 64 * 32 : v;
}

size_t score_smem_bytes(const ScoreConfig& cfg, int mark_words);
// Blocks of the persistent scoring kernel that fit on the device at once.
int score_grid(const ScoreConfig& cfg, int mark_words);
// Launch the persistent scorer with min(grid, a.n) blocks; *a.next must be
// zero when it starts.
cudaError_t launch_score(const ScoreArgs& a, const ScoreConfig& cfg, int grid, cudaStream_t s);
// Add a scoring kernel node to graph g after the given dependencies; the
// caller resets *a.next before the node runs.
cudaError_t add_score_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                           const ScoreArgs& a, const ScoreConfig& cfg, int grid, cudaGraphNode_t* out);

// M2M GICP refinement (Sec. IV-A): one launch refines the hypotheses of one
// job; each block holds its hypothesis' source cloud in a slot of `src`.
struct GicpArgs {
    Job job;                  // poses = input poses (device); costs unused
    long long n;
    int zcap_words;
    int* err;
    unsigned* next;           // hypothesis counter, zeroed before the launch
    unsigned* smask;          // slot mask, (slots + 31) / 32 words, zero when idle
    int slots;
    float4* src;              // slots x src_cap x (point, normal)
    int src_cap;
    unsigned long long* vcache;  // slots x vstride vertex records, or nullptr
    long long vstride;
    const float4* nrm;        // observed normal per pixel (H*W)
    int max_iters, min_corr;
    float epsilon, stop_rot, stop_trans;
    float* poses_out;         // n*12 (device)
    int32_t* info;            // n*2 (device) or nullptr
};

size_t gicp_smem_bytes(int zcap_words);
int gicp_grid(int zcap_words);
cudaError_t launch_gicp(const GicpArgs& a, int grid, cudaStream_t s);
// Observed normal per pixel from central differences of the depth image.
cudaError_t launch_obs_normals(const DevScene& sc, int normal_jump, float4* nrm, cudaStream_t s);

// ADD (symmetric 0) / ADD-S (1) of n pose pairs over a mesh's vertices.
cudaError_t launch_add_s(const float4* verts, int n_verts, const float* poses, const float* poses_true,
                         long long n, int symmetric, double* out, cudaStream_t s);

// Observation build (voxel hash over I).
struct BuildBuffers {
    // scratch (freed after the build)
    int32_t* slot_of_pixel;   // H*W
    unsigned long long* keys; // table capacity
    uint32_t* count;          // table capacity
    uint32_t* cursor;         // table capacity
    uint32_t* start;          // table capacity
    int* n_valid;             // 2: valid points, occupied cells
    // outputs (owned by the scene)
    float4* lab;              // H*W
    float4* pxyz;             // H*W
    float4* pts;              // n_points capacity (H*W)
    uint4* table;             // table capacity
};
cudaError_t launch_build(const DevScene& sc, const BuildBuffers& b, uint32_t table_cap,
                         const uint8_t* rgb_dev, int* err, cudaStream_t s);
cudaError_t launch_compact_table(const uint4* big, uint32_t cap_big, uint4* small, uint32_t cap_small,
                                 int* err, cudaStream_t s);
// Bounding box of the observed points' hash cells: bounds = (min x, y, z, max x, y, z).
cudaError_t launch_cell_bounds(const DevScene& sc, int* bounds, cudaStream_t s);
// Fill sc.near_bits (zeroed) through the occupancy bitmap occ (zeroed, same size).
cudaError_t launch_near_cells(const DevScene& sc, uint32_t* occ, uint32_t* near_bits, cudaStream_t s);
// Dense cell index over the near-cell box: cell_start (n_cells + 1 words;
// the last one is written by the caller) and the points re-sorted by cell
// into out.  count and cursor (n_cells words each) and tile_sums
// ((n_cells + 1023) / 1024 words) are zeroed scratch.
cudaError_t launch_dense_cells(const DevScene& sc, uint32_t* count, uint32_t* cursor, uint32_t* tile_sums,
                               uint32_t* cell_start, float4* out, cudaStream_t s);

// Argmin of J = J_o + J_r (ties to the lowest id / index).  The kernel
// launches at most kBestMaxBlocks blocks; each leaves three 64-bit words
// (packed cost, id, index) in `partial`.
constexpr int kBestMaxBlocks = 1024;
struct BestArgs {
    const int32_t* costs;
    const unsigned long long* ids;  // or nullptr
    long long n;
    long long* best_index;
    int32_t* best_cost;
    unsigned long long* partial;    // scratch: 3 words per block, 3 * kBestMaxBlocks words
    unsigned int* ticket;           // scratch: 1 word, zero on entry, zero on exit
    unsigned long long* key;        // or nullptr: the winner as (J << 32) | low 32 bits of its id
};
int best_blocks(long long n);
cudaError_t launch_best(const BestArgs& a, cudaStream_t s);

cudaError_t init_device_tables(cudaStream_t s);

// 6-DoF pose proposals (Sec. V-B): z range of a labelled box, then the poses.
struct ProposalArgs {
    DevScene sc;
    int label;
    int box[4];
    int M, N, K;
    float centre[3];          // object-frame centre of the mesh's bounding box
    unsigned* zr;             // device: [z_min, z_max] (0.1 mm), reduced by the first kernel
    int32_t* z_out;           // optional copy of zr (device), or nullptr
    float* poses;             // device, M*N*K*12
};
cudaError_t launch_proposals(const ProposalArgs& a, cudaStream_t s);

}  // namespace perch
