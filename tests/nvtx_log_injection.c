/* NVTX injection library for the tests: every range pushed by the process is written,
 * one name per line, to the file named by TDLZ_TEST_NVTX_LOG.  Loaded by the NVTX
 * headers of the library under test when NVTX_INJECTION64_PATH points to it. */
#include <nvtx3/nvToolsExt.h>
#include <stdio.h>
#include <stdlib.h>

static FILE *g_log = NULL;

static int log_push(const char *name) {
  if (g_log && name) {
    fprintf(g_log, "%s\n", name);
    fflush(g_log);
  }
  return 0;
}

static int log_pop(void) { return 0; }

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
  const NvtxExportTableCallbacks *cb =
      (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
  NvtxFunctionTable table = NULL;
  unsigned int size = 0;
  if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) || !table)
    return 0;
  const char *path = getenv("TDLZ_TEST_NVTX_LOG");
  g_log = path ? fopen(path, "w") : NULL;
  if (NVTX_CBID_CORE_RangePushA < size)
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)log_push;
  if (NVTX_CBID_CORE_RangePop < size)
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)log_pop;
  return 1;
}
