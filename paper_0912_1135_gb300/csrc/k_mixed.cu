// Mixed mode orchestration (sliced bfloat16 tensor-core products). Placeholder until
// the sliced GEMM lands: every entry reports RTPROJ_EUNSUPPORTED.
#include "rtproj_internal.cuh"

namespace rtp {
size_t mixed_bytes(int64_t, int64_t, int64_t, int64_t, const rtproj_opts&) { return 0; }
rtproj_status mixed_bind(rtproj_ctx*, char*, size_t) { return RTPROJ_EUNSUPPORTED; }
rtproj_status mixed_prepare_a(rtproj_ctx*) { return RTPROJ_EUNSUPPORTED; }
rtproj_status mixed_sketch(rtproj_ctx*, uint64_t, int64_t, double*, int64_t) { return RTPROJ_EUNSUPPORTED; }
rtproj_status mixed_gram(rtproj_ctx*) { return RTPROJ_EUNSUPPORTED; }
rtproj_status mixed_project(rtproj_ctx*, const double*, int64_t, int, double*, int64_t, double*, int64_t, double*,
                            int64_t) {
    return RTPROJ_EUNSUPPORTED;
}
}  // namespace rtp
