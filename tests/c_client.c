/* A plain C client of libmbc (include/mbc.h): plans the proton correlator from the
 * library's operator library, reports the plan statistics and, on a device, evaluates
 * C(t) from fields read from a file through both the device and the host-buffer entry
 * points.  Used by tests/test_c_client.py to show that the ABI works from C alone.
 *
 * usage: c_client <device> [<fields file> <T> <V3>]
 *   fields file: U then D, complex double [T][V3][12][12] each (raw, little endian)
 * output lines: "terms <n>", "canonical <n>", "guard <site threshold> <slice tolerance>"
 * and "shape <threads> <blocks per site> <leaf batch>" of an MBC_PREC_FP32 plan after
 * setting them, then "C <t> <re> <im>", "H <t> <re> <im>" (FP64, device and host-buffer
 * results) and "F <t> <re> <im>" (FP32 with guards) when a device is given.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "mbc.h"

static int die(mbc_ctx* ctx, const char* what) {
    fprintf(stderr, "%s: %s\n", what, ctx ? mbc_last_error(ctx) : "");
    return 1;
}

int main(int argc, char** argv) {
    if (argc < 2) return 2;
    const int device = atoi(argv[1]);
    mbc_ctx* ctx = NULL;
    if (mbc_create(&ctx, device) != MBC_OK) return die(NULL, "mbc_create");

    int n_u, n_d, n_free;
    int64_t n_terms;
    if (mbc_operator_terms(MBC_OP_PROTON, &n_u, &n_d, &n_free, &n_terms, NULL, NULL, NULL, NULL, NULL) != MBC_OK)
        return die(ctx, "mbc_operator_terms");
    int8_t* idx = (int8_t*)malloc((size_t)n_terms * (n_u + n_d));
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)n_terms);
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (n_free + 1));
    double* proj = (double*)malloc(sizeof(double) * 2 * n_free * n_free);
    double scale = 0.0;
    if (!idx || !w || !off || !proj) return 3;
    if (mbc_operator_terms(MBC_OP_PROTON, &n_u, &n_d, &n_free, &n_terms, idx, w, off, proj, &scale) != MBC_OK)
        return die(ctx, "mbc_operator_terms");
    printf("terms %lld\n", (long long)n_terms);

    mbc_problem pr;
    pr.n_u = n_u; pr.n_d = n_d; pr.n_free = n_free;
    pr.snk_idx = idx; pr.snk_w = w; pr.snk_off = off;
    pr.src_idx = idx; pr.src_w = w; pr.src_off = off;
    pr.proj = proj;
    pr.scale[0] = scale; pr.scale[1] = 0.0;
    mbc_plan* plan = NULL;
    if (mbc_plan_create(ctx, &pr, MBC_ALGO_EGRAPH, MBC_PREC_FP64, &plan) != MBC_OK) return die(ctx, "mbc_plan_create");
    mbc_plan_info info;
    if (mbc_plan_get_info(plan, &info) != MBC_OK) return die(ctx, "mbc_plan_get_info");
    printf("canonical %lld\n", (long long)info.canonical_terms);
    mbc_plan* p32 = NULL;
    if (mbc_plan_create(ctx, &pr, MBC_ALGO_EGRAPH, MBC_PREC_FP32, &p32) != MBC_OK) return die(ctx, "FP32 plan");
    if (mbc_plan_set_guard(p32, 3.0, 5e-7) != MBC_OK) return die(ctx, "mbc_plan_set_guard");
    double g_site = 0.0, g_slice = 0.0;
    if (mbc_plan_get_guard(p32, &g_site, &g_slice) != MBC_OK) return die(ctx, "mbc_plan_get_guard");
    printf("guard %g %g\n", g_site, g_slice);
    mbc_schedule sh = {384, 1, 2};
    if (mbc_set_schedule(p32, &sh) != MBC_OK) return die(ctx, "mbc_set_schedule");
    if (mbc_get_schedule(p32, &sh) != MBC_OK) return die(ctx, "mbc_get_schedule");
    printf("shape %d %d %d\n", sh.threads, sh.blocks_per_sm, sh.sites_per_unit);

    if (device >= 0 && argc >= 5) {
        const int T = atoi(argv[3]);
        const int64_t V3 = atoll(argv[4]);
        const size_t n = (size_t)T * V3 * 288;            /* doubles per flavour */
        double* h = (double*)malloc(sizeof(double) * 2 * n);
        FILE* f = fopen(argv[2], "rb");
        if (!h || !f || fread(h, sizeof(double), 2 * n, f) != 2 * n) return 4;
        fclose(f);
        void *U = NULL, *D = NULL, *C = NULL;
        if (cudaMalloc(&U, sizeof(double) * n) != cudaSuccess || cudaMalloc(&D, sizeof(double) * n) != cudaSuccess ||
            cudaMalloc(&C, sizeof(double) * 2 * T) != cudaSuccess)
            return 5;
        cudaMemcpy(U, h, sizeof(double) * n, cudaMemcpyHostToDevice);
        cudaMemcpy(D, h + n, sizeof(double) * n, cudaMemcpyHostToDevice);
        if (mbc_correlator(plan, U, D, 1, T, V3, C, NULL, NULL) != MBC_OK) return die(ctx, "mbc_correlator");
        double* c = (double*)malloc(sizeof(double) * 2 * T);
        if (cudaMemcpy(c, C, sizeof(double) * 2 * T, cudaMemcpyDeviceToHost) != cudaSuccess) return 6;
        for (int t = 0; t < T; ++t) printf("C %d %.17g %.17g\n", t, c[2 * t], c[2 * t + 1]);
        if (mbc_correlator_host(plan, h, h + n, 1, T, V3, c, NULL) != MBC_OK) return die(ctx, "mbc_correlator_host");
        for (int t = 0; t < T; ++t) printf("H %d %.17g %.17g\n", t, c[2 * t], c[2 * t + 1]);
        if (mbc_correlator(p32, U, D, 1, T, V3, C, NULL, NULL) != MBC_OK) return die(ctx, "FP32 mbc_correlator");
        if (cudaMemcpy(c, C, sizeof(double) * 2 * T, cudaMemcpyDeviceToHost) != cudaSuccess) return 6;
        for (int t = 0; t < T; ++t) printf("F %d %.17g %.17g\n", t, c[2 * t], c[2 * t + 1]);
        cudaFree(U); cudaFree(D); cudaFree(C);
        free(c);
        free(h);
    }
    mbc_plan_destroy(p32);
    mbc_plan_destroy(plan);
    mbc_destroy(ctx);
    free(idx); free(w); free(off); free(proj);
    return 0;
}
