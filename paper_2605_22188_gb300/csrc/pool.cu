// C entry points of the support pool (App. G layout; see pool.h).
#include <string.h>

#include <new>

#include "kglm.h"
#include "pool.h"

extern "C" {

kglm_status kglm_pool_create(int32_t p, kglm_pool** out) {
    if (!out) return KGLM_EINVAL;
    *out = nullptr;
    if (p <= 0) return KGLM_EINVAL;
    kglm_pool* q = new (std::nothrow) kglm_pool();
    if (!q) return KGLM_ENOMEM;
    q->p = p;
    *out = q;
    return KGLM_OK;
}

kglm_status kglm_pool_insert(kglm_pool* q, int32_t len, const int32_t* seq, const double* coef, double objective,
                             int64_t* record) {
    if (!q || len < 0 || (len > 0 && (!seq || !coef))) return KGLM_EINVAL;
    std::vector<int> s(seq, seq + len);
    for (int a : s)
        if (a < 0 || a >= q->p) return KGLM_EINVAL;
    std::vector<int> sorted(s);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return KGLM_EINVAL;
    try {
        const int64_t r = q->insert(s, std::vector<double>(coef, coef + len), objective);
        if (record) *record = r;
    } catch (const std::bad_alloc&) {
        return KGLM_ENOMEM;
    }
    return KGLM_OK;
}

kglm_status kglm_pool_size(const kglm_pool* q, int64_t* records, int64_t* trie_nodes, int64_t* coef_len) {
    if (!q) return KGLM_EINVAL;
    if (records) *records = (int64_t)q->leaf.size();
    if (trie_nodes) *trie_nodes = (int64_t)q->parent.size();
    if (coef_len) *coef_len = (int64_t)q->coef.size();
    return KGLM_OK;
}

kglm_status kglm_pool_read(const kglm_pool* q, int64_t* offsets, double* coef, double* objective, int32_t* leaf,
                           int32_t* parent, int32_t* label) {
    if (!q) return KGLM_EINVAL;
    const size_t R = q->leaf.size(), V = q->parent.size();
    if (offsets) memcpy(offsets, q->off.data(), sizeof(int64_t) * (R + 1));
    if (coef && !q->coef.empty()) memcpy(coef, q->coef.data(), sizeof(double) * q->coef.size());
    if (objective && R) memcpy(objective, q->obj.data(), sizeof(double) * R);
    for (size_t r = 0; r < R && leaf; ++r) leaf[r] = q->leaf[r];
    for (size_t v = 0; v < V; ++v) {
        if (parent) parent[v] = q->parent[v];
        if (label) label[v] = q->label[v];
    }
    return KGLM_OK;
}

kglm_status kglm_pool_support(const kglm_pool* q, int64_t record, int32_t* labels, int32_t* len) {
    if (!q || record < 0 || record >= (int64_t)q->leaf.size()) return KGLM_EINVAL;
    const std::vector<int> s = q->path(q->leaf[record]);
    if (labels) std::copy(s.begin(), s.end(), labels);
    if (len) *len = (int32_t)s.size();
    return KGLM_OK;
}

kglm_status kglm_pool_filter(kglm_pool* q, double threshold, int64_t keep_best) {
    if (!q || keep_best < 0) return KGLM_EINVAL;
    try {
        q->filter(threshold, keep_best);
    } catch (const std::bad_alloc&) {
        return KGLM_ENOMEM;
    }
    return KGLM_OK;
}

void kglm_pool_destroy(kglm_pool* q) { delete q; }

}  // extern "C"
