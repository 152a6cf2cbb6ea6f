/*
 * Exhaustive 2-domination number of the cylinder P_n x C_m, straight from
 * the graph definition (Section 1): S is 2-dominating when every vertex
 * outside S has at least two neighbours in S.  No words, no transfer matrix:
 * this is an independent pin for the oracle's enumerator, arc rule and the
 * min-diagonal readout of Theorem 2.  Subsets are tried by increasing size
 * (Gosper's next-combination step), so the first size that works is gamma_2.
 *
 * Vertex (i, j), i in [0, n) along the path, j in [0, m) around the cycle,
 * has bit i*m + j.  Needs n*m <= 30.
 */
#include <stdint.h>

static int popc(uint32_t x) { return __builtin_popcount(x); }

int brute_gamma2(int n, int m)
{
    int V = n * m;
    if (n < 1 || m < 3 || V > 30) return -1;
    uint32_t nb[30];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            uint32_t b = 0;
            if (i > 0) b |= 1u << ((i - 1) * m + j);
            if (i + 1 < n) b |= 1u << ((i + 1) * m + j);
            b |= 1u << (i * m + (j + 1) % m);
            b |= 1u << (i * m + (j + m - 1) % m);
            nb[i * m + j] = b;
        }
    uint32_t full = (V == 32) ? 0xFFFFFFFFu : ((1u << V) - 1u);
    for (int k = 0; k <= V; ++k) {
        if (k == 0) continue; /* V >= 3, the empty set never works */
        uint32_t s = (1u << k) - 1u;
        while (s <= full) {
            int ok = 1;
            for (int v = 0; v < V && ok; ++v)
                if (!((s >> v) & 1u) && popc(s & nb[v]) < 2) ok = 0;
            if (ok) return k;
            /* next subset with the same popcount */
            uint32_t c = s & (0u - s), r = s + c;
            if (r == 0 || r > full) break;
            s = (((r ^ s) >> 2) / c) | r;
        }
    }
    return -1;
}
