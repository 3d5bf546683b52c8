/* A plain C caller of the library (no Python): one 16 x 16 image holding a
 * square ring of foreground around a 4 x 4 hole, analysed and hole-filled
 * through include/ccl.h. Expected: three nodes (exterior 0, the ring, the
 * hole), Euler number 0, the hole absorbed by the ring when filled.
 * Exit status: 0 ok, 1 wrong result, 2 no CUDA device (the library reports
 * CCL_ERR_CUDA rather than falling back). */
#include <stdio.h>
#include <string.h>
#include <cuda_runtime_api.h>
#include "ccl.h"

#define W 16
#define H 16

int main(void) {
    unsigned char img[H][W];
    memset(img, 0, sizeof img);
    for (int y = 4; y < 12; ++y)
        for (int x = 4; x < 12; ++x) img[y][x] = (y < 6 || y >= 10 || x < 6 || x >= 10) ? 1 : 0;

    ccl_ctx *ctx = NULL;
    ccl_status st = ccl_create(&ctx, W, H, W);
    if (st == CCL_ERR_CUDA) {
        printf("no device: %s\n", ccl_status_string(st));
        return 2;
    }
    if (st != CCL_OK) return 1;
    const int64_t cap = ccl_node_capacity(W, H);
    unsigned char *d_img;
    int32_t *d_fg, *d_bg, *d_parent, *d_counts, *d_map, *d_fparent;
    int64_t *d_feat, *d_ffeat;
    cudaMalloc((void **)&d_img, sizeof img);
    cudaMalloc((void **)&d_fg, sizeof(int32_t) * W * H);
    cudaMalloc((void **)&d_bg, sizeof(int32_t) * W * H);
    cudaMalloc((void **)&d_parent, sizeof(int32_t) * cap);
    cudaMalloc((void **)&d_counts, sizeof(int32_t) * 4);
    cudaMalloc((void **)&d_feat, sizeof(int64_t) * CCL_F_COUNT * cap);
    cudaMalloc((void **)&d_map, sizeof(int32_t) * cap);
    cudaMalloc((void **)&d_fparent, sizeof(int32_t) * cap);
    cudaMalloc((void **)&d_ffeat, sizeof(int64_t) * CCL_F_COUNT * cap);
    cudaMemcpy(d_img, img, sizeof img, cudaMemcpyHostToDevice);

    st = ccl_analyze(ctx, d_img, d_fg, d_bg, d_parent, d_feat, d_counts, 0);
    if (st != CCL_OK) return 1;
    int32_t n = 0, nf = 0, nb = 0;
    int64_t euler = 0;
    st = ccl_get_counts(ctx, &n, &nf, &nb);
    if (st != CCL_OK || ccl_get_euler(ctx, &euler) != CCL_OK) return 1;
    st = ccl_fill_holes(ctx, INT64_MAX, d_map, d_ffeat, d_fparent, 0);
    if (st != CCL_OK || ccl_get_counts(ctx, NULL, NULL, NULL) != CCL_OK) return 1;

    int32_t parent[3], map[3], fg[H][W];
    int64_t area[3], farea[3];
    cudaMemcpy(parent, d_parent, sizeof parent, cudaMemcpyDeviceToHost);
    cudaMemcpy(map, d_map, sizeof map, cudaMemcpyDeviceToHost);
    cudaMemcpy(area, d_feat + CCL_F_AREA * cap, sizeof area, cudaMemcpyDeviceToHost);
    cudaMemcpy(farea, d_ffeat + CCL_F_AREA * cap, sizeof farea, cudaMemcpyDeviceToHost);
    cudaMemcpy(fg, d_fg, sizeof fg, cudaMemcpyDeviceToHost);
    printf("nodes %d fg %d bg %d euler %lld parent %d %d %d area %lld %lld %lld map %d %d %d filled ring area %lld\n",
           n, nf, nb, (long long)euler, parent[0], parent[1], parent[2], (long long)area[0], (long long)area[1],
           (long long)area[2], map[0], map[1], map[2], (long long)farea[1]);
    const int ok = n == 3 && nf == 1 && nb == 2 && euler == 0 && parent[0] == -1 && parent[1] == 0 &&
                   parent[2] == 1 && area[0] == 256 - 64 && area[1] == 48 && area[2] == 16 && map[0] == 0 &&
                   map[1] == 1 && map[2] == 1 && farea[1] == 64 && fg[4][4] == 1 && fg[0][0] == -1;
    ccl_destroy(ctx);
    return ok ? 0 : 1;
}
