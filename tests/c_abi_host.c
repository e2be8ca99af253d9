/* A plain C11 caller of libsrp: includes include/srp.h, links the shared
 * library and exercises the host-only entry points (no GPU needed): option
 * defaults, design instantiation (a hinge rotation), the host BVH build
 * (two-call pattern, every triangle in exactly one leaf), the proxy's
 * parameter count and an error status with its message.  Exit status 0 and
 * "c-abi ok" on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "srp.h"

#define CHECK(cond, what)                                      \
    do {                                                       \
        if (!(cond)) {                                         \
            fprintf(stderr, "FAILED: %s (%s)\n", what, #cond); \
            return 1;                                          \
        }                                                      \
    } while (0)

int main(void) {
    srp_trace_opts o;
    srp_trace_opts_default(&o);
    CHECK(o.rays_x == 1024 && o.rays_y == 1024 && o.max_bounces == 1 && o.pressure == 1.0, "trace defaults");
    srp_orbit_opts oo;
    srp_orbit_opts_default(&oo);
    CHECK(oo.dt == 60.0 && oo.n_steps == 1440 && oo.model == SRP_FM_NONE, "orbit defaults");

    /* hinge along +z through the origin: (1, 0, 0) turns to (0, 1, 0) */
    const float vin[6] = {1.0f, 0.0f, 0.0f, 2.0f, 0.0f, 0.0f};
    const int32_t vh[2] = {0, -1};
    const double hinge[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 1.0};
    const double ang[1] = {acos(-1.0) / 2.0};
    float vout[6];
    CHECK(srp_design_instantiate(vin, 2, vh, hinge, ang, 1, vout) == SRP_OK, "instantiate");
    CHECK(fabsf(vout[0]) < 1e-6f && fabsf(vout[1] - 1.0f) < 1e-6f && vout[3] == 2.0f, "hinge rotation");

    /* a unit cube: 8 vertices, 12 triangles */
    const float cv[24] = {0, 0, 0, 1, 0, 0, 1, 1, 0, 0, 1, 0, 0, 0, 1, 1, 0, 1, 1, 1, 1, 0, 1, 1};
    const int32_t ct[36] = {0, 2, 1, 0, 3, 2, 4, 5, 6, 4, 6, 7, 0, 1, 5, 0, 5, 4,
                            1, 2, 6, 1, 6, 5, 2, 3, 7, 2, 7, 6, 3, 0, 4, 3, 4, 7};
    for (int width = 4; width <= 8; width += 4) {
        int64_t nf = 0;
        int32_t nn = 0;
        CHECK(srp_build_bvh_host(cv, 8, ct, 12, width, NULL, &nf, NULL, &nn) == SRP_OK, "bvh sizes");
        CHECK(nn >= 1 && nf == (int64_t)nn * (width == 4 ? 32 : 64), "bvh node floats");
        float* nodes = (float*)malloc(sizeof(float) * (size_t)nf);
        int32_t order[12];
        CHECK(nodes != NULL, "malloc");
        CHECK(srp_build_bvh_host(cv, 8, ct, 12, width, nodes, &nf, order, &nn) == SRP_OK, "bvh build");
        int seen[12] = {0};
        for (int k = 0; k < 12; ++k) {
            CHECK(order[k] >= 0 && order[k] < 12, "leaf order index");
            seen[order[k]]++;
        }
        /* every leaf range [first, first + count) of every node, summed */
        int covered[12] = {0};
        for (int32_t n = 0; n < nn; ++n) {
            int32_t code[8];
            memcpy(code, nodes + (size_t)n * (width == 4 ? 32 : 64) + 6 * width, sizeof(int32_t) * (size_t)width);
            for (int c = 0; c < width; ++c) {
                if (code[c] >= 0 || nodes[(size_t)n * (width == 4 ? 32 : 64) + c] > nodes[(size_t)n * (width == 4 ? 32 : 64) + width + c])
                    continue; /* inner child or empty slot (lo > hi) */
                const int32_t leaf = ~code[c], first = leaf >> 3, count = (leaf & 7) + 1;
                CHECK(first >= 0 && first + count <= 12, "leaf range");
                for (int k = first; k < first + count; ++k) covered[k]++;
            }
        }
        for (int k = 0; k < 12; ++k) CHECK(seen[k] == 1 && covered[k] == 1, "each triangle in one leaf");
        free(nodes);
    }

    int64_t np = 0;
    CHECK(srp_mlp_param_count(&np) == SRP_OK && np == 19 * 256 + 256 + 3 * (256 * 256 + 256) + 256 * 6 + 6,
          "proxy parameter count");

    /* an invalid width is refused with a message */
    int64_t nf = 0;
    int32_t nn = 0;
    CHECK(srp_build_bvh_host(cv, 8, ct, 12, 5, NULL, &nf, NULL, &nn) == SRP_EINVAL, "bad width refused");
    CHECK(srp_last_error() != NULL && strlen(srp_last_error()) > 0, "error message");
    printf("c-abi ok\n");
    return 0;
}
