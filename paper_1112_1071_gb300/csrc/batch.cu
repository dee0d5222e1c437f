// Batched models (hrt_batch_*): many contexts advanced together, one Lucy iteration each.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/hrt.h"

struct hrt_batch {
    std::vector<hrt_ctx*> models;
    std::vector<int> done;
};

extern "C" {

int hrt_batch_create(hrt_batch** out, hrt_ctx* const* models, int n) {
    if (!out || !models || n < 1) return HRT_EINVAL;
    hrt_batch* b = new hrt_batch();
    b->models.assign(models, models + n);
    b->done.assign(n, 0);
    *out = b;
    return HRT_OK;
}

int hrt_batch_destroy(hrt_batch* b) {
    if (!b) return HRT_EINVAL;
    delete b;
    return HRT_OK;
}

int hrt_batch_run(hrt_batch* b, const int64_t* n_packets, int max_iter, const hrt_run_params* params,
                  hrt_iter_stats* per_model_out, int* iterations_run) {
    if (!b || !n_packets || max_iter < 0) return HRT_EINVAL;
    int iters = 0;
    for (int it = 0; it < max_iter; ++it) {
        bool any = false;
        for (size_t m = 0; m < b->models.size(); ++m) {
            if (b->done[m]) continue;
            hrt_iter_stats st;
            int rc = hrt_run_iteration(b->models[m], n_packets[m], params, &st);
            if (rc != HRT_OK) return rc;
            if (per_model_out) per_model_out[m] = st;
            if (st.converged) b->done[m] = 1;
            any = true;
        }
        if (!any) break;
        ++iters;
    }
    if (iterations_run) *iterations_run = iters;
    return HRT_OK;
}

int hrt_batch_tune(hrt_batch* b, const int64_t* n_packets) {
    if (!b || !n_packets) return HRT_EINVAL;
    return HRT_OK;
}

}  // extern "C"
