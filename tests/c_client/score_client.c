/* A plain C client of libperch (no Python, no torch): reads one scene, one
 * mesh and its pose hypotheses from a binary file, scores them through the C
 * ABI in host mode, takes the argmin, and writes the costs.  Test
 * infrastructure: it shows that include/perch.h and libperch.so are usable
 * from C alone.
 *
 * Input (little endian): int32 W, H, n_verts, n_tris, n_poses; float fx, fy,
 * cx, cy, delta, tau_c, vol_r, vol_h; int32 color_check; then depth uint16
 * [H*W], rgb uint8 [H*W*3], verts float [n_verts*3], vertex rgb uint8
 * [n_verts*3], tris int32 [n_tris*3], poses float [n_poses*12].
 * Output: costs int32 [n_poses*2], then int64 best index and int32 best cost.
 * Exit status 0 on success, else the failing step's number. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "perch.h"

static int read_all(FILE *f, void *p, size_t bytes)
{
    return fread(p, 1, bytes, f) == bytes;
}

int main(int argc, char **argv)
{
    if (argc != 3) {
        fprintf(stderr, "usage: %s input.bin output.bin\n", argv[0]);
        return 1;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in) return 2;
    int32_t hdr[5];
    float fl[8];
    int32_t color_check;
    if (!read_all(in, hdr, sizeof hdr) || !read_all(in, fl, sizeof fl) ||
        !read_all(in, &color_check, sizeof color_check))
        return 3;
    const int32_t W = hdr[0], H = hdr[1], nv = hdr[2], nt = hdr[3], n = hdr[4];
    if (W < 1 || H < 1 || nv < 1 || nt < 1 || n < 1) return 4;
    uint16_t *depth = malloc(sizeof(uint16_t) * (size_t)W * H);
    uint8_t *rgb = malloc((size_t)W * H * 3);
    float *verts = malloc(sizeof(float) * 3 * (size_t)nv);
    uint8_t *vrgb = malloc(3 * (size_t)nv);
    int32_t *tris = malloc(sizeof(int32_t) * 3 * (size_t)nt);
    float *poses = malloc(sizeof(float) * 12 * (size_t)n);
    int32_t *costs = malloc(sizeof(int32_t) * 2 * (size_t)n);
    if (!depth || !rgb || !verts || !vrgb || !tris || !poses || !costs) return 5;
    if (!read_all(in, depth, sizeof(uint16_t) * (size_t)W * H) || !read_all(in, rgb, (size_t)W * H * 3) ||
        !read_all(in, verts, sizeof(float) * 3 * (size_t)nv) || !read_all(in, vrgb, 3 * (size_t)nv) ||
        !read_all(in, tris, sizeof(int32_t) * 3 * (size_t)nt) || !read_all(in, poses, sizeof(float) * 12 * (size_t)n))
        return 6;
    fclose(in);

    perch_ctx *ctx = NULL;
    if (perch_create(&ctx, 0, 0) != PERCH_OK) return 7;
    perch_params p;
    perch_default_params(&p);
    p.delta_m = fl[4];
    p.tau_c = fl[5];
    p.color_check = color_check;
    int32_t scene = -1, mesh = -1;
    if (perch_set_observation(ctx, depth, rgb, NULL, W, H, fl[0], fl[1], fl[2], fl[3], &p, &scene) != PERCH_OK) {
        fprintf(stderr, "%s\n", perch_last_error(ctx));
        return 8;
    }
    if (perch_load_mesh(ctx, verts, vrgb, nv, tris, nt, fl[6], fl[7], &mesh) != PERCH_OK) return 9;
    if (perch_score_hypotheses(ctx, scene, mesh, -1, NULL, poses, n, costs, NULL) != PERCH_OK) {
        fprintf(stderr, "%s\n", perch_last_error(ctx));
        return 10;
    }
    int64_t best_index = -1;
    int32_t best_cost = -1;
    if (perch_best(ctx, costs, NULL, n, &best_index, &best_cost, NULL) != PERCH_OK) return 11;
    perch_destroy(ctx);

    FILE *out = fopen(argv[2], "wb");
    if (!out) return 12;
    fwrite(costs, sizeof(int32_t), 2 * (size_t)n, out);
    fwrite(&best_index, sizeof best_index, 1, out);
    fwrite(&best_cost, sizeof best_cost, 1, out);
    fclose(out);
    free(depth); free(rgb); free(verts); free(vrgb); free(tris); free(poses); free(costs);
    return 0;
}
