/*
 * A plain C client of the C ABI (include/tvlp.h): no Python, no PyTorch.
 * Reads a, e, gs (float32, binary) for one batch, runs lp_tv_forward_f32 and
 * lp_tv_backward_f32 with LP_BWD_REUSE_FORWARD on device buffers it
 * allocates with the CUDA runtime, and writes s, ge, ga, gzi back out.
 *
 *   tvlp_client B T M in_dir out_dir
 * in_dir holds a.bin [B][T][M], e.bin [B][T], gs.bin [B][T], zi.bin [B][M];
 * out_dir receives s.bin, ge.bin, ga.bin, gzi.bin.  Exit status 0 on
 * success; any error prints the library's message and exits 1.
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "tvlp.h"

static void *read_file(const char *dir, const char *name, size_t bytes) {
    char path[1024];
    snprintf(path, sizeof path, "%s/%s", dir, name);
    FILE *f = fopen(path, "rb");
    if (!f) return NULL;
    void *buf = malloc(bytes);
    size_t got = buf ? fread(buf, 1, bytes, f) : 0;
    fclose(f);
    if (got != bytes) {
        free(buf);
        return NULL;
    }
    return buf;
}

static int write_file(const char *dir, const char *name, const void *buf, size_t bytes) {
    char path[1024];
    snprintf(path, sizeof path, "%s/%s", dir, name);
    FILE *f = fopen(path, "wb");
    if (!f) return 0;
    size_t put = fwrite(buf, 1, bytes, f);
    fclose(f);
    return put == bytes;
}

#define CHECK_LP(x)                                                        \
    do {                                                                   \
        int rc_ = (x);                                                     \
        if (rc_ != LP_OK) {                                                \
            fprintf(stderr, "%s: %s\n", #x, lp_strerror(rc_));             \
            return 1;                                                      \
        }                                                                  \
    } while (0)
#define CHECK_CUDA(x)                                                      \
    do {                                                                   \
        if ((x) != cudaSuccess) {                                          \
            fprintf(stderr, "%s failed\n", #x);                            \
            return 1;                                                      \
        }                                                                  \
    } while (0)

int main(int argc, char **argv) {
    if (argc != 6) {
        fprintf(stderr, "usage: %s B T M in_dir out_dir\n", argv[0]);
        return 2;
    }
    const int B = atoi(argv[1]), M = atoi(argv[3]);
    const int64_t T = atoll(argv[2]);
    const size_t nbt = (size_t)B * (size_t)T, nbtm = nbt * (size_t)M, nbm = (size_t)B * (size_t)M;
    float *ha = read_file(argv[4], "a.bin", nbtm * 4), *he = read_file(argv[4], "e.bin", nbt * 4);
    float *hgs = read_file(argv[4], "gs.bin", nbt * 4), *hzi = read_file(argv[4], "zi.bin", nbm * 4);
    if (!ha || !he || !hgs || !hzi) {
        fprintf(stderr, "cannot read the inputs\n");
        return 1;
    }
    const size_t wsb = lp_tv_workspace_bytes(B, T, M, 0, LP_DTYPE_F32);
    float *a, *e, *gs, *zi, *s, *ge, *ga, *gzi;
    void *ws;
    CHECK_CUDA(cudaMalloc((void **)&a, nbtm * 4));
    CHECK_CUDA(cudaMalloc((void **)&e, nbt * 4));
    CHECK_CUDA(cudaMalloc((void **)&gs, nbt * 4));
    CHECK_CUDA(cudaMalloc((void **)&zi, nbm * 4));
    CHECK_CUDA(cudaMalloc((void **)&s, nbt * 4));
    CHECK_CUDA(cudaMalloc((void **)&ge, nbt * 4));
    CHECK_CUDA(cudaMalloc((void **)&ga, nbtm * 4));
    CHECK_CUDA(cudaMalloc((void **)&gzi, nbm * 4));
    CHECK_CUDA(cudaMalloc(&ws, wsb > 0 ? wsb : 256));
    CHECK_CUDA(cudaMemcpy(a, ha, nbtm * 4, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(e, he, nbt * 4, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(gs, hgs, nbt * 4, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(zi, hzi, nbm * 4, cudaMemcpyHostToDevice));
    cudaStream_t st;
    CHECK_CUDA(cudaStreamCreate(&st));
    CHECK_LP(lp_tv_forward_f32(B, T, M, a, e, zi, s, NULL, 0, LP_ALGO_CHUNKED, ws, wsb, st));
    CHECK_LP(lp_tv_backward_f32(B, T, M, gs, a, s, zi, ge, ga, gzi, 0, LP_ALGO_CHUNKED, LP_BWD_REUSE_FORWARD, ws,
                                wsb, st));
    CHECK_CUDA(cudaStreamSynchronize(st));
    if (lp_tv_device_status(0) != 0) {
        fprintf(stderr, "device status %d\n", lp_tv_device_status(0));
        return 1;
    }
    float *out = malloc(nbtm * 4);
    if (!out) return 1;
    CHECK_CUDA(cudaMemcpy(out, s, nbt * 4, cudaMemcpyDeviceToHost));
    if (!write_file(argv[5], "s.bin", out, nbt * 4)) return 1;
    CHECK_CUDA(cudaMemcpy(out, ge, nbt * 4, cudaMemcpyDeviceToHost));
    if (!write_file(argv[5], "ge.bin", out, nbt * 4)) return 1;
    CHECK_CUDA(cudaMemcpy(out, ga, nbtm * 4, cudaMemcpyDeviceToHost));
    if (!write_file(argv[5], "ga.bin", out, nbtm * 4)) return 1;
    CHECK_CUDA(cudaMemcpy(out, gzi, nbm * 4, cudaMemcpyDeviceToHost));
    if (!write_file(argv[5], "gzi.bin", out, nbm * 4)) return 1;
    printf("tvlp_client ok: %s\n", lp_version());
    return 0;
}
