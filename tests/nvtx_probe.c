/* A minimal NVTX injection library for the tests: it records every range
 * push (with its name) and pop of the process in the file named by
 * SKEI_TEST_NVTX_LOG.  Loaded by NVTX itself when NVTX_INJECTION64_PATH
 * names it. */
#include <nvtx3/nvToolsExt.h>
#include <stdio.h>
#include <stdlib.h>

static FILE *g_log;

static int probe_push(const char *message) {
  if (g_log) {
    fprintf(g_log, "push %s\n", message ? message : "");
    fflush(g_log);
  }
  return 0;
}

static int probe_pop(void) {
  if (g_log) {
    fprintf(g_log, "pop\n");
    fflush(g_log);
  }
  return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
  const NvtxExportTableCallbacks *cb =
      (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
  NvtxFunctionTable table = 0;
  unsigned int size = 0;
  const char *path = getenv("SKEI_TEST_NVTX_LOG");
  if (!cb || !path || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size)) return 0;
  if (size <= NVTX_CBID_CORE_RangePop) return 0;
  g_log = fopen(path, "w");
  *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)probe_push;
  *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)probe_pop;
  return g_log != 0;
}
