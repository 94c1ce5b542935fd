// Kernel-activity trace through CUPTI (a profiling aid, not part of the step).
// trace_start() enables concurrent-kernel and memset activity records;
// trace_stop(path) flushes them and writes one line per record:
//   start_ns end_ns stream_id name
// Built on demand by paper_2108_04435_gb300/trace.py.
#include <cupti.h>
#include <stdio.h>
#include <stdlib.h>

#include <string>
#include <vector>

namespace {

struct Rec {
    unsigned long long start, end;
    unsigned stream;
    std::string name;
};
std::vector<Rec> g_recs;

void CUPTIAPI buffer_requested(uint8_t** buf, size_t* size, size_t* max_records) {
    *size = 16u << 20;
    *buf = (uint8_t*)aligned_alloc(8, *size);
    *max_records = 0;
}

void CUPTIAPI buffer_completed(CUcontext, uint32_t, uint8_t* buf, size_t, size_t valid) {
    CUpti_Activity* r = nullptr;
    while (cuptiActivityGetNextRecord(buf, valid, &r) == CUPTI_SUCCESS) {
        if (r->kind == CUPTI_ACTIVITY_KIND_CONCURRENT_KERNEL || r->kind == CUPTI_ACTIVITY_KIND_KERNEL) {
            const auto* k = (const CUpti_ActivityKernel10*)r;
            g_recs.push_back({k->start, k->end, k->streamId, k->name ? k->name : "?"});
        } else if (r->kind == CUPTI_ACTIVITY_KIND_MEMSET) {
            const auto* m = (const CUpti_ActivityMemset4*)r;
            g_recs.push_back({m->start, m->end, m->streamId, "memset"});
        }
    }
    free(buf);
}

}  // namespace

extern "C" int trace_start() {
    g_recs.clear();
    if (cuptiActivityRegisterCallbacks(buffer_requested, buffer_completed) != CUPTI_SUCCESS) return -1;
    if (cuptiActivityEnable(CUPTI_ACTIVITY_KIND_CONCURRENT_KERNEL) != CUPTI_SUCCESS) return -2;
    cuptiActivityEnable(CUPTI_ACTIVITY_KIND_MEMSET);
    return 0;
}

extern "C" int trace_stop(const char* path) {
    cuptiActivityFlushAll(1);
    cuptiActivityDisable(CUPTI_ACTIVITY_KIND_CONCURRENT_KERNEL);
    cuptiActivityDisable(CUPTI_ACTIVITY_KIND_MEMSET);
    FILE* f = fopen(path, "w");
    if (!f) return -1;
    for (const Rec& r : g_recs) fprintf(f, "%llu %llu %u %s\n", r.start, r.end, r.stream, r.name.c_str());
    fclose(f);
    return (int)g_recs.size();
}
