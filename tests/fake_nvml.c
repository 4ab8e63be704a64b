/* A stand-in for libnvidia-ml with the entry points libsy resolves: two devices,
 * a fixed list of supported clocks, and SM-clock locks that only change this
 * file's state.  Every lock and reset call is appended to a log the tests read;
 * an injected return code makes one entry point fail.  Test infrastructure: it
 * lets the clock-control paths run on a machine without a GPU and without ever
 * changing a real device's settings. */
#include <stdio.h>
#include <string.h>

typedef int ret_t;
typedef void* device_t;

enum { OK = 0, INVALID_ARGUMENT = 2, NOT_FOUND = 6, INSUFFICIENT_SIZE = 7 };
enum { CLOCK_GRAPHICS = 0, CLOCK_SM = 1, CLOCK_MEM = 2 };

static const unsigned kMem[2] = {3996, 1598};
static const unsigned kSmAtMem0[11] = {2070, 1965, 1860, 1755, 1650, 1545, 1440, 1335, 1230, 1125, 1020};
static const unsigned kSmAtMem1[3] = {1410, 1200, 990};
static const unsigned kSmMax = 2070;

static int g_dev[2];
static unsigned g_lock_min[2], g_lock_max[2];
static unsigned g_mem_now = 3996;
static char g_log[8192];
static char g_fail_name[128];
static ret_t g_fail_code;

static void logf_(const char* s) {
    size_t n = strlen(g_log);
    if (n + strlen(s) + 1 < sizeof g_log) strcat(g_log, s);
}

static ret_t injected(const char* name) {
    return strcmp(name, g_fail_name) == 0 ? g_fail_code : OK;
}

static int index_of(device_t d) {
    if (d == (device_t)&g_dev[0]) return 0;
    if (d == (device_t)&g_dev[1]) return 1;
    return -1;
}

static ret_t list_out(const unsigned* v, unsigned n, unsigned* count, unsigned* out) {
    if (!count) return INVALID_ARGUMENT;
    if (!out || *count < n) {
        *count = n;
        return INSUFFICIENT_SIZE;
    }
    memcpy(out, v, n * sizeof(unsigned));
    *count = n;
    return OK;
}

/* ---- inspection and injection (not NVML) ---- */
const char* fake_nvml_log(void) { return g_log; }
void fake_nvml_clear(void) { g_log[0] = 0; }
void fake_nvml_fail(const char* name, int code) {
    snprintf(g_fail_name, sizeof g_fail_name, "%s", name ? name : "");
    g_fail_code = code;
}
void fake_nvml_set_mem_clock(unsigned mhz) { g_mem_now = mhz; }
void fake_nvml_locked(int dev, unsigned* lo, unsigned* hi) {
    *lo = g_lock_min[dev];
    *hi = g_lock_max[dev];
}

/* ---- the NVML entry points ---- */
ret_t nvmlInit_v2(void) { return injected("nvmlInit_v2"); }
ret_t nvmlShutdown(void) { return OK; }

ret_t nvmlDeviceGetHandleByIndex_v2(unsigned index, device_t* d) {
    if (index > 1 || !d) return INVALID_ARGUMENT;
    *d = (device_t)&g_dev[index];
    return injected("nvmlDeviceGetHandleByIndex_v2");
}

ret_t nvmlDeviceGetHandleByPciBusId_v2(const char* bus, device_t* d) {
    (void)bus;
    if (!d) return INVALID_ARGUMENT;
    *d = (device_t)&g_dev[0];
    return OK;
}

ret_t nvmlDeviceGetIndex(device_t d, unsigned* index) {
    int i = index_of(d);
    if (i < 0 || !index) return INVALID_ARGUMENT;
    *index = (unsigned)i;
    return OK;
}

ret_t nvmlDeviceGetTotalEnergyConsumption(device_t d, unsigned long long* mj) {
    if (index_of(d) < 0 || !mj) return INVALID_ARGUMENT;
    *mj = 1000;
    return OK;
}

ret_t nvmlDeviceGetClockInfo(device_t d, int type, unsigned* mhz) {
    int i = index_of(d);
    if (i < 0 || !mhz) return INVALID_ARGUMENT;
    if (type == CLOCK_MEM) *mhz = g_mem_now;
    else *mhz = g_lock_max[i] ? g_lock_max[i] : kSmMax;
    return injected("nvmlDeviceGetClockInfo");
}

ret_t nvmlDeviceGetMaxClockInfo(device_t d, int type, unsigned* mhz) {
    if (index_of(d) < 0 || !mhz) return INVALID_ARGUMENT;
    *mhz = type == CLOCK_MEM ? kMem[0] : kSmMax;
    return OK;
}

ret_t nvmlDeviceGetSupportedMemoryClocks(device_t d, unsigned* count, unsigned* mhz) {
    if (index_of(d) < 0) return INVALID_ARGUMENT;
    return list_out(kMem, 2, count, mhz);
}

ret_t nvmlDeviceGetSupportedGraphicsClocks(device_t d, unsigned mem, unsigned* count, unsigned* mhz) {
    if (index_of(d) < 0) return INVALID_ARGUMENT;
    if (mem == kMem[0]) return list_out(kSmAtMem0, 11, count, mhz);
    if (mem == kMem[1]) return list_out(kSmAtMem1, 3, count, mhz);
    return NOT_FOUND;
}

ret_t nvmlDeviceSetGpuLockedClocks(device_t d, unsigned lo, unsigned hi) {
    int i = index_of(d);
    char buf[64];
    if (i < 0) return INVALID_ARGUMENT;
    snprintf(buf, sizeof buf, "lock:%d:%u:%u;", i, lo, hi);
    logf_(buf);
    ret_t r = injected("nvmlDeviceSetGpuLockedClocks");
    if (r == OK) {
        g_lock_min[i] = lo;
        g_lock_max[i] = hi;
    }
    return r;
}

ret_t nvmlDeviceResetGpuLockedClocks(device_t d) {
    int i = index_of(d);
    char buf[32];
    if (i < 0) return INVALID_ARGUMENT;
    snprintf(buf, sizeof buf, "reset:%d;", i);
    logf_(buf);
    g_lock_min[i] = g_lock_max[i] = 0;
    return injected("nvmlDeviceResetGpuLockedClocks");
}
