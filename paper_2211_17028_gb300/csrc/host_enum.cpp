// Kept assignments of the level-l expansion (Sec. IV, Algorithm 1) and their
// canonical ranks.
//
// Canonical order: level u ascending; within a level the site tuple
// p_1 < ... < p_u lexicographically; within a site tuple the factor tuple
// lexicographically over each site's kept non-dominant factors (all three,
// i = 1, 2, 3, unless zero-rank pruning removed some).  With m_s kept factors
// at site s, the number of level-u terms is the elementary symmetric sum
// e_u(m_0, ..., m_{N-1}), which for m_s = 3 is C(N,u) 3^u (Theorem 1).
#include "nqs_internal.h"

namespace nqs {

void TermIndex::build(const std::vector<int>& m_per_site, int lvl) {
    m = m_per_site;
    N = (int)m.size();
    level = lvl;
    E.assign(level + 1, std::vector<uint64_t>(N + 1, 0));
    for (int a = 0; a <= N; ++a) E[0][a] = 1;
    for (int j = 1; j <= level; ++j)
        for (int a = N - 1; a >= 0; --a) E[j][a] = E[j][a + 1] + (uint64_t)m[a] * E[j - 1][a + 1];
    level_offset.assign(level + 2, 0);
    for (int u = 0; u <= level; ++u) level_offset[u + 1] = level_offset[u] + E[u][0];
    total = level_offset[level + 1];
}

uint64_t TermIndex::rank(int k, const int* sites, const int* fpos) const {
    uint64_t r = level_offset[k];
    uint64_t prefix = 1;
    int prev = -1;
    for (int j = 0; j < k; ++j) {
        // tuples equal on the first j sites with a smaller site at position j
        for (int x = prev + 1; x < sites[j]; ++x) r += prefix * (uint64_t)m[x] * E[k - 1 - j][x + 1];
        prefix *= (uint64_t)m[sites[j]];
        prev = sites[j];
    }
    uint64_t radix = 1, idx = 0;
    for (int j = k - 1; j >= 0; --j) {
        idx += (uint64_t)fpos[j] * radix;
        radix *= (uint64_t)m[sites[j]];
    }
    return r + idx;
}

}  // namespace nqs
