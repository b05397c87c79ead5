// Loading and launching instrumented PTX (Sec. V-E: the transformed module is loaded into
// the worker-owned context). The CUDA runtime's library API JIT-compiles the PTX for the
// current device; the guard's module globals are pointed at the table and the log
// before any launch, and a launch is refused until they are.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>

#include "agile_internal.h"

struct agile_module {
    cudaLibrary_t lib = nullptr;
    bool guarded = false;   // carries the guard's module globals
    bool aperture = false;  // guarded by the aperture rule: needs no table
    bool bound = false;
};

extern "C" {

int agile_module_load(const char *ptx, agile_module_t **out) {
    if (ptx == nullptr || out == nullptr) return AGILE_ERR_INVALID_ARG;
    *out = nullptr;
    agile_module *m = new (std::nothrow) agile_module;
    if (m == nullptr) return AGILE_ERR_NOMEM;
    thread_local char errlog[8192];   // per thread: loads may run concurrently
    errlog[0] = '\0';
    cudaJitOption opt[2] = {cudaJitErrorLogBuffer, cudaJitErrorLogBufferSizeBytes};
    void *val[2] = {errlog, (void *)(uintptr_t)sizeof errlog};
    cudaError_t e = cudaLibraryLoadData(&m->lib, ptx, opt, val, 2, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
        std::string msg = std::string("cudaLibraryLoadData (JIT): ") + errlog;
        agile::set_cuda_error((int)e, msg.substr(0, 200).c_str());
        delete m;
        return AGILE_ERR_CUDA;
    }
    void *g = nullptr;
    size_t b = 0;
    m->guarded = cudaLibraryGetGlobal(&g, &b, m->lib, "__agile_guard_table") == cudaSuccess;
    (void)cudaGetLastError();
    m->aperture = m->guarded &&
                  cudaLibraryGetGlobal(&g, &b, m->lib, "__agile_aperture_mode") == cudaSuccess;
    (void)cudaGetLastError();
    *out = m;
    return AGILE_OK;
}

int agile_module_bind(agile_module_t *m, const agile_dev_table_t *tbl, void *d_log, void *stream) {
    if (m == nullptr || !m->guarded || (tbl == nullptr && !m->aperture)) return AGILE_ERR_INVALID_ARG;
    if (d_log != nullptr && ((uintptr_t)d_log & 15) != 0) return AGILE_ERR_ALIGN;
    void *g_tbl = nullptr, *g_log = nullptr;
    size_t b1 = 0, b2 = 0;
    AGILE_CUDA_TRY(cudaLibraryGetGlobal(&g_tbl, &b1, m->lib, "__agile_guard_table"));
    AGILE_CUDA_TRY(cudaLibraryGetGlobal(&g_log, &b2, m->lib, "__agile_guard_log"));
    if (b1 != 8 || b2 != 8) return AGILE_ERR_PTX_UNSUPPORTED;
    // The header sits at the start of the table's device buffer.
    uint64_t vals[2] = {tbl ? (uint64_t)(uintptr_t)agile::table_buffer(*tbl) : 0, (uint64_t)(uintptr_t)d_log};
    cudaStream_t st = (cudaStream_t)stream;
    AGILE_CUDA_TRY(cudaMemcpyAsync(g_tbl, &vals[0], 8, cudaMemcpyHostToDevice, st));
    AGILE_CUDA_TRY(cudaMemcpyAsync(g_log, &vals[1], 8, cudaMemcpyHostToDevice, st));
    AGILE_CUDA_TRY(cudaStreamSynchronize(st));
    m->bound = true;
    return AGILE_OK;
}

int agile_module_launch(agile_module_t *m, const char *name, uint32_t grid, uint32_t block,
                        void **args, void *stream) {
    if (m == nullptr || name == nullptr || grid == 0 || block == 0 || block > 1024)
        return AGILE_ERR_INVALID_ARG;
    if (m->guarded && !m->bound) return AGILE_ERR_INVALID_ARG;   // guard not pointed at a table
    cudaKernel_t k = nullptr;
    cudaError_t e = cudaLibraryGetKernel(&k, m->lib, name);
    if (e != cudaSuccess) {
        agile::set_cuda_error((int)e, "cudaLibraryGetKernel");
        return AGILE_ERR_NOT_FOUND;
    }
    AGILE_CUDA_TRY(cudaLaunchKernel((const void *)k, dim3(grid), dim3(block), args, 0,
                                    (cudaStream_t)stream));
    return AGILE_OK;
}

void agile_module_unload(agile_module_t *m) {
    if (m == nullptr) return;
    if (m->lib) cudaLibraryUnload(m->lib);
    delete m;
}

}  // extern "C"
