/* A minimal NVTX tool for the tests: loaded by the NVTX runtime of libaidw.so
 * through NVTX_INJECTION64_PATH, it replaces the push and pop of named ranges
 * with functions that append one line per event to the file named by
 * AIDW_NVTX_LOG ("push <name>" or "pop"), so that a test can check which
 * ranges a library call opened and that each was closed. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE *log_file;
static int depth;

static int record_push(const char *name)
{
    if (log_file) {
        fprintf(log_file, "push %s\n", name ? name : "");
        fflush(log_file);
    }
    return depth++;
}

static int record_pop(void)
{
    if (log_file) {
        fputs("pop\n", log_file);
        fflush(log_file);
    }
    return --depth;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_export_table)
{
    const char *path = getenv("AIDW_NVTX_LOG");
    if (!path || !(log_file = fopen(path, "a"))) return 0;
    const NvtxExportTableCallbacks *cb =
        (const NvtxExportTableCallbacks *)get_export_table(NVTX_ETID_CALLBACKS);
    if (!cb || !cb->GetModuleFunctionTable) return 0;
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    if (!cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) ||
        size <= NVTX_CBID_CORE_RangePop)
        return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)record_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)record_pop;
    return 1;
}
