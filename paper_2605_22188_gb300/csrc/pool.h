// Support pool of a Rashomon-set collection (§4.5) in the compact layout of
// App. G: a trie whose non-root nodes carry one feature index each (the path
// from the root to a record's leaf lists the record's support in insertion
// order), and the records' coefficients in one vector c cut by offsets o
// (o_0 = 0, o_m = o_{m-1} + |S_m|), so that record m's coefficients are
// c[o_{m-1} .. o_m) in the order of its path labels.  Host-side structure.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <limits>
#include <map>
#include <set>
#include <vector>

struct kglm_pool {
    int p = 0;
    // trie: node 0 is the root; node v > 0 has parent[v] and label[v]
    std::vector<int> parent{-1}, label{-1};
    std::map<std::pair<int, int>, int> child;   // (parent, label) -> node
    // records, in insertion order
    std::vector<int> leaf;
    std::vector<double> obj;
    std::vector<int64_t> off{0};
    std::vector<double> coef;
    std::set<std::vector<int>> held;            // sorted supports present

    // Path labels of a leaf, root first.
    std::vector<int> path(int v) const {
        std::vector<int> s;
        for (; v > 0; v = parent[v]) s.push_back(label[v]);
        return std::vector<int>(s.rbegin(), s.rend());
    }
    // Adds a record unless its support is already held; returns its index or -1.
    int64_t insert(const std::vector<int>& seq, const std::vector<double>& c, double objective) {
        std::vector<int> key(seq);
        std::sort(key.begin(), key.end());
        if (held.count(key)) return -1;
        int v = 0;
        for (int a : seq) {
            auto it = child.find({v, a});
            if (it == child.end()) {
                parent.push_back(v);
                label.push_back(a);
                const int u = (int)parent.size() - 1;
                child[{v, a}] = u;
                v = u;
            } else {
                v = it->second;
            }
        }
        held.insert(key);
        leaf.push_back(v);
        obj.push_back(objective);
        coef.insert(coef.end(), c.begin(), c.end());
        off.push_back((int64_t)coef.size());
        return (int64_t)leaf.size() - 1;
    }
    // Keeps the records with objective <= threshold and, if keep > 0, only the
    // keep best of those (ties to the earlier record); the kept records are
    // re-inserted in their original order, so the trie holds no dead branches.
    void filter(double threshold, int64_t keep) {
        std::vector<int64_t> idx;
        for (int64_t r = 0; r < (int64_t)leaf.size(); ++r)
            if (obj[r] <= threshold) idx.push_back(r);
        if (keep > 0 && (int64_t)idx.size() > keep) {
            std::vector<int64_t> by(idx);
            std::stable_sort(by.begin(), by.end(), [&](int64_t a, int64_t b) { return obj[a] < obj[b]; });
            by.resize(keep);
            std::sort(by.begin(), by.end());
            idx.swap(by);
        }
        if (idx.size() == leaf.size()) return;
        kglm_pool q;
        q.p = p;
        for (int64_t r : idx) {
            const std::vector<double> c(coef.begin() + off[r], coef.begin() + off[r + 1]);
            q.insert(path(leaf[r]), c, obj[r]);
        }
        *this = std::move(q);
    }
    // N-th best objective held (+inf with fewer than N records).
    double nth_best(int64_t N) const {
        if (N <= 0 || (int64_t)obj.size() < N) return std::numeric_limits<double>::infinity();
        std::vector<double> o(obj);
        std::nth_element(o.begin(), o.begin() + (N - 1), o.end());
        return o[N - 1];
    }
};
