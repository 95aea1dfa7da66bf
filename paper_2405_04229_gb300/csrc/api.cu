// Status strings, error reporting and device checks of the C ABI.
#include <stdio.h>

#include "common.cuh"

namespace cs {

static thread_local char g_last_error[512] = "";

void set_last_error(const char* where, cudaError_t e) {
    snprintf(g_last_error, sizeof g_last_error, "%s: %s (%s)", where, cudaGetErrorName(e),
             cudaGetErrorString(e));
}

// The kernels are built for sm_103a only: require compute capability 10.3.
cs_status check_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        if (e != cudaSuccess) set_last_error("cudaGetDeviceCount", e);
        return CS_ERR_NO_DEVICE;
    }
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) {
        snprintf(g_last_error, sizeof g_last_error, "device %d has compute capability %d.%d, need 10.3",
                 dev, major, minor);
        return CS_ERR_NO_DEVICE;
    }
    return CS_OK;
}

int device_sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace cs

extern "C" const char* cs_status_string(cs_status s) {
    switch (s) {
    case CS_OK: return "CS_OK";
    case CS_ERR_INVALID_ARG: return "CS_ERR_INVALID_ARG";
    case CS_ERR_CUDA: return "CS_ERR_CUDA";
    case CS_ERR_CAPACITY: return "CS_ERR_CAPACITY";
    case CS_ERR_TIMEOUT: return "CS_ERR_TIMEOUT";
    case CS_ERR_DOMAIN: return "CS_ERR_DOMAIN";
    case CS_ERR_NO_DEVICE: return "CS_ERR_NO_DEVICE";
    }
    return "CS_ERR_UNKNOWN";
}

extern "C" const char* cs_last_error(void) { return cs::g_last_error; }

extern "C" cs_status cs_device_sm_count(int* n_sm) {
    if (!n_sm) return CS_ERR_INVALID_ARG;
    cs_status st = cs::check_device();
    if (st != CS_OK) return st;
    *n_sm = cs::device_sm_count();
    return CS_OK;
}

extern "C" void cs_opts_default(cs_opts* o) {
    if (!o) return;
    o->bunch = 1;
    o->s_max = 1.0;
    o->seg_base = 0;
    o->device_ptrs = 0;
    o->accumulate = 0;
    o->block_threads = 0;
    o->blocks_per_sm = 0;
    o->surrogate = nullptr;
    o->lv1_metric = CS_LV1_OFF;
    o->lv1_a = 0.0;
    o->lv1_b = 0.0;
    o->lv1_centre[0] = o->lv1_centre[1] = o->lv1_centre[2] = 0.0;
    o->lv1_radius = 0.0;
    o->lv1_dropped = nullptr;
    o->lv3 = 0;
    o->lv3_centre[0] = o->lv3_centre[1] = o->lv3_centre[2] = 0.0;
    o->lv3_radius = o->lv3_margin = 0.0;
    o->tracer = CS_TRACER_TABLES;
    o->tracer_dh = 10.0;
    o->emission = CS_EMIT_CHERENKOV;
    o->fl_n_lines = 0;
    o->fl_lines_nm = nullptr;
    o->fl_yield_per_mev = nullptr;
    o->fl_dedx = 2.2;
    o->tc_poll_limit = 0;
    o->exact_queue = 0;
}
