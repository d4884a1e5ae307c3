// libperch M2M GICP refinement of hypotheses (Sec. IV-A "Parallel M2M
// GICP"): scratch management and the C entry points; the kernels are in
// perch_kernels.cu.
#include "perch_host.cuh"

#include <algorithm>

using namespace perch_host;

namespace {

// Grow a scratch buffer of X (after every earlier run that used X).
perch_status grow(perch_ctx* c, ScoreScratch& X, void** buf, size_t* have, size_t need)
{
    if (need <= *have) return PERCH_OK;
    cudaEventSynchronize(X.last);
    dfree(c, *buf);
    *buf = nullptr;
    *have = 0;
    perch_status st = dalloc(c, need, buf);
    if (st == PERCH_OK) *have = need;
    return st;
}

// Launch the GICP refinement of one job on stream st, after every earlier run
// that used X (they share the counter, the slot pool and the caches).
perch_status run_gicp(perch_ctx* c, ScoreScratch& X, const perch::Job& J, const perch_gicp_params& gp,
                      const float4* nrm, float* poses_out, int32_t* info, cudaStream_t st)
{
    if (J.n == 0) return PERCH_OK;
    if (J.n > 0xFFFFFFF0ll) return fail(c, PERCH_E_INVALID, "more than 2^32 hypotheses in one call");
    int dev = 0, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int zcap = c->cfg.zcap_words;
    while (perch::gicp_smem_bytes(zcap) > (size_t)max_optin && zcap > 1024) zcap /= 2;
    const int grid = perch::gicp_grid(zcap);
    if (grid <= 0) {
        cudaGetLastError();
        return fail(c, PERCH_E_CUDA, "refinement kernel does not fit on the device");
    }
    const long long s = J.sc.stride;
    const long long lattice = ((J.roi[2] - J.roi[0] + s - 1) / s) * ((J.roi[3] - J.roi[1] + s - 1) / s);
    long long cap = gp.max_source_points > 0 ? gp.max_source_points : 65536;
    cap = std::max(1ll, std::min(cap, lattice));
    perch_status stt = grow(c, X, &X.src, &X.src_bytes, (size_t)grid * (size_t)cap * 2 * sizeof(float4));
    if (stt != PERCH_OK) return stt;
    long long vstride = 0;
    if (J.sc.W <= 1023 && J.sc.H <= 1023) {
        vstride = ((long long)J.m.n_verts + 31) / 32 * 32;
        stt = grow(c, X, &X.vcache, &X.vcache_bytes, (size_t)grid * vstride * sizeof(unsigned long long));
        if (stt != PERCH_OK) return stt;
    }
    const size_t words = 1 + ((size_t)grid + 31) / 32;
    if (words > X.next_words) {
        size_t have = X.next_words * sizeof(unsigned);
        void* p = X.next;
        stt = grow(c, X, &p, &have, std::max<size_t>(words, 64) * sizeof(unsigned));
        X.next = (unsigned*)p;
        X.next_words = have / sizeof(unsigned);
        if (stt != PERCH_OK) return stt;
    }
    perch::GicpArgs a{};
    a.job = J;
    a.n = J.n;
    a.zcap_words = zcap;
    a.err = c->d_err;
    a.next = X.next;
    a.smask = X.next + 1;
    a.slots = grid;
    a.src = (float4*)X.src;
    a.src_cap = (int)cap;
    a.vcache = vstride ? (unsigned long long*)X.vcache : nullptr;
    a.vstride = vstride;
    a.nrm = nrm;
    a.max_iters = gp.max_iterations;
    a.min_corr = gp.min_correspondences;
    a.epsilon = gp.epsilon;
    a.stop_rot = gp.stop_rotation_rad;
    a.stop_trans = gp.stop_translation_m;
    a.poses_out = poses_out;
    a.info = info;
    cudaError_t e = cudaStreamWaitEvent(st, X.last, 0);
    if (!e) e = cudaMemsetAsync(X.next, 0, words * sizeof(unsigned), st);
    if (!e) e = perch::launch_gicp(a, grid, st);
    if (!e) e = cudaEventRecord(X.last, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "refinement launch");
    return PERCH_OK;
}

}  // namespace

extern "C" {

perch_status perch_default_gicp_params(perch_gicp_params* p)
{
    if (!p) return PERCH_E_INVALID;
    p->max_iterations = 10;
    p->epsilon = 1e-3f;
    p->normal_max_jump_units = 200;
    p->min_correspondences = 6;
    p->stop_rotation_rad = 1e-5f;
    p->stop_translation_m = 1e-5f;
    p->max_source_points = 0;
    return PERCH_OK;
}

perch_status perch_refine_hypotheses(perch_ctx* c, int32_t scene_id, int32_t mesh_id, int32_t label,
                                     const int32_t* roi, const float* poses, int64_t n,
                                     const perch_gicp_params* params, float* poses_out, int32_t* info,
                                     void* cuda_stream)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (n < 0) return fail(c, PERCH_E_INVALID, "n < 0");
    if (n == 0) return PERCH_OK;
    if (!poses || !poses_out || !params) return fail(c, PERCH_E_INVALID, "null poses, poses_out or params");
    const perch_gicp_params gp = *params;
    if (gp.max_iterations < 0 || gp.max_iterations > 1000)
        return fail(c, PERCH_E_INVALID, "max_iterations must be in [0, 1000]");
    if (!finite(gp.epsilon) || !(gp.epsilon > 0.0f) || !(gp.epsilon < 1.0f))
        return fail(c, PERCH_E_INVALID, "epsilon must be in (0, 1)");
    if (gp.normal_max_jump_units < 0 || gp.min_correspondences < 1 || gp.max_source_points < 0)
        return fail(c, PERCH_E_INVALID, "normal_max_jump_units, min_correspondences or max_source_points out of range");
    if (!finite(gp.stop_rotation_rad) || !finite(gp.stop_translation_m) || gp.stop_rotation_rad < 0.0f ||
        gp.stop_translation_m < 0.0f)
        return fail(c, PERCH_E_INVALID, "stop thresholds must be finite and >= 0");
    perch_status st = refuse_while_serving(c);
    if (st != PERCH_OK) return st;
    DeviceGuard g(c->device);
    Range r("perch: GICP refinement");
    perch::Job J;
    int mw;
    st = make_job(c, scene_id, mesh_id, label, roi, poses, nullptr, n, &J, &mw, nullptr, nullptr);
    if (st != PERCH_OK) return st;
    J.sc.jo_mode = 0;
    // observed normals of the scene for this jump threshold (made once, synchronously)
    SceneRec& S = c->scenes[scene_id];
    if (!S.nrm || S.nrm_jump != gp.normal_max_jump_units) {
        cudaEventSynchronize(c->plain.last);
        if (!S.nrm && (st = dalloc(c, (size_t)S.ds.W * S.ds.H * sizeof(float4), &S.nrm)) != PERCH_OK) return st;
        cudaError_t e = perch::launch_obs_normals(S.ds, gp.normal_max_jump_units, (float4*)S.nrm, c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
        if (e) return cuda_fail(c, e, "observed normals");
        S.nrm_jump = gp.normal_max_jump_units;
    }
    const float4* nrm = (const float4*)S.nrm;
    if (cuda_stream) {
        st = run_gicp(c, c->plain, J, gp, nrm, poses_out, info, (cudaStream_t)cuda_stream);
        return st != PERCH_OK ? st : note_async_use(c, scene_id, mesh_id, (cudaStream_t)cuda_stream);
    }
    const long long chunk = 1 << 18;
    const long long k0 = std::min<long long>(n, chunk);
    if ((st = ensure_stage(c, (size_t)k0 * (48 + 48 + 8))) != PERCH_OK) return st;
    float* d_in = (float*)c->stage;
    float* d_out = (float*)((char*)c->stage + (size_t)k0 * 48);
    int32_t* d_info = (int32_t*)((char*)c->stage + (size_t)k0 * 96);
    for (long long off = 0; off < n; off += chunk) {
        const long long k = std::min(chunk, n - off);
        cudaError_t e = cudaMemcpyAsync(d_in, poses + 12 * off, k * 48, cudaMemcpyHostToDevice, c->stream);
        if (e) return cuda_fail(c, e, "perch_refine_hypotheses upload");
        perch::Job Jk = J;
        Jk.poses = d_in;
        Jk.n = k;
        if ((st = run_gicp(c, c->plain, Jk, gp, nrm, d_out, d_info, c->stream)) != PERCH_OK) return st;
        e = cudaMemcpyAsync(poses_out + 12 * off, d_out, k * 48, cudaMemcpyDeviceToHost, c->stream);
        if (!e && info) e = cudaMemcpyAsync(info + 2 * off, d_info, k * 8, cudaMemcpyDeviceToHost, c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
        if (e) return cuda_fail(c, e, "perch_refine_hypotheses");
    }
    return check_device_error(c);
}

}  // extern "C"
