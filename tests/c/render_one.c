/*
 * A plain C client of the vgr ABI (no Python, no PyTorch): builds a 3-node
 * LoD tree (a root and two leaf Gaussians), renders one 64 x 64 frame into
 * host memory and prints the cut and the brightest pixel.  The test suite
 * compiles and links it against include/vgr.h and libvgr.so on any machine,
 * and runs it where a GPU is present.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "vgr.h"

static int check(vgr_status s, const char* what) {
    if (s != VGR_OK) {
        fprintf(stderr, "%s: status %d: %s\n", what, (int)s, vgr_last_error());
        return 1;
    }
    return 0;
}

int main(void) {
    /* root (node 0) with two leaf children, BFS order, children contiguous */
    const uint32_t parent[3] = {0xFFFFFFFFu, 0, 0};
    const uint32_t first_child[3] = {1, 0, 0};
    const uint8_t n_child[3] = {2, 0, 0};
    const float mean[9] = {0.0f, 0.0f, 5.0f, -0.3f, 0.0f, 5.0f, 0.3f, 0.0f, 5.0f};
    const float cov6[18] = {0.04f, 0, 0, 0.04f, 0, 0.04f, 0.01f, 0, 0, 0.01f, 0, 0.01f, 0.01f, 0, 0, 0.01f, 0, 0.01f};
    const float opacity[3] = {0.8f, 0.7f, 0.7f};
    const float sh[9] = {0.5f, 0.5f, 0.5f, 1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 1.0f}; /* degree 0: DC per node */
    const float radius2[3] = {1.0f, 0.09f, 0.09f};
    vgr_scene_desc d = {3, 0, parent, first_child, n_child, mean, cov6, opacity, sh, radius2, VGR_STORE_FP32, NULL};

    vgr_hierarchy* h = NULL;
    vgr_view* v = NULL;
    if (check(vgr_load_hierarchy(&d, &h), "load")) return 1;
    vgr_view_opts o;
    vgr_default_view_opts(&o);
    if (check(vgr_create_view(h, &o, &v), "view")) return 1;

    /* camera at the origin looking down +z; tau small enough that the root expands */
    vgr_camera cam = {{1, 0, 0, 0, 1, 0, 0, 0, 1}, {0, 0, 0}, 60.0f, 60.0f, 32.0f, 32.0f, 64, 64, 0.2f};
    float* img = (float*)malloc(64 * 64 * 3 * sizeof(float));
    vgr_frame fr;
    if (!img || check(vgr_render_frame_host(v, &cam, 1.0f, img, &fr), "render")) return 1;
    float best = 0.0f;
    for (int i = 0; i < 64 * 64 * 3; ++i)
        if (img[i] > best) best = img[i];
    printf("cut %u nodes, visible %u, pairs %llu, brightest %.4f\n", fr.cut_count, fr.stats.visible_count,
           (unsigned long long)fr.stats.pair_count, best);
    free(img);
    vgr_destroy_view(v);
    vgr_free_hierarchy(h);
    return fr.cut_count == 2 && best > 0.1f ? 0 : 2;
}
