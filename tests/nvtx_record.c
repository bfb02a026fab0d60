/* A minimal NVTX injection library for the tests: loaded by NVTX when
 * NVTX_INJECTION64_PATH names it, it appends one line per domain range push
 * ("push <domain> <message>") and pop ("pop <domain>") to the file named by
 * HC_NVTX_LOG.  Only the three domain calls the library uses are hooked. */
#define NVTX_NO_IMPL
#include <nvtx3/nvToolsExt.h>

#include <pthread.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

struct nvtxDomainRegistration_st {
    char name[64];
};

static pthread_mutex_t g_lock = PTHREAD_MUTEX_INITIALIZER;
static FILE* g_log;

static void log_line(const char* a, const char* b, const char* c) {
    pthread_mutex_lock(&g_lock);
    if (g_log) {
        fprintf(g_log, "%s %s%s%s\n", a, b, c ? " " : "", c ? c : "");
        fflush(g_log);
    }
    pthread_mutex_unlock(&g_lock);
}

static nvtxDomainHandle_t NVTX_API domain_create(const char* name) {
    nvtxDomainHandle_t d = (nvtxDomainHandle_t)calloc(1, sizeof(*d));
    if (d) snprintf(d->name, sizeof(d->name), "%s", name ? name : "");
    return d;
}

static int NVTX_API range_push(nvtxDomainHandle_t d, const nvtxEventAttributes_t* a) {
    const char* msg = (a && a->messageType == NVTX_MESSAGE_TYPE_ASCII) ? a->message.ascii : "?";
    log_line("push", d ? d->name : "-", msg);
    return 0;
}

static int NVTX_API range_pop(nvtxDomainHandle_t d) {
    log_line("pop", d ? d->name : "-", NULL);
    return 0;
}

int NVTX_API InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
    const char* path = getenv("HC_NVTX_LOG");
    g_log = path ? fopen(path, "a") : NULL;
    const NvtxExportTableCallbacks* cb =
        (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
    if (!cb) return 0;
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    if (!cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE2, &table, &size) || !table) return 0;
    if (size <= NVTX_CBID_CORE2_DomainCreateA) return 0;
    *table[NVTX_CBID_CORE2_DomainCreateA] = (NvtxFunctionPointer)domain_create;
    *table[NVTX_CBID_CORE2_DomainRangePushEx] = (NvtxFunctionPointer)range_push;
    *table[NVTX_CBID_CORE2_DomainRangePop] = (NvtxFunctionPointer)range_pop;
    return 1;
}
