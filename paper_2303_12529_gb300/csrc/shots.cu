// Mask fracturing shot count (Sec. II-C.3): the number of rectangles a mask is
// fractured into. Reading: the minimum number of non-overlapping axis-aligned
// rectangles whose union is the mask (a minimum rectangle partition). Host code: the
// count is a graph matching per connected piece of the mask, not per-pixel work.
//
// For a rectilinear polygon with v vertices and h holes, the minimum partition has
// v / 2 + h - g - 1 rectangles, g being the largest set of pairwise non-intersecting
// "good chords" (segments inside the polygon joining two reflex vertices on one grid
// line); horizontal chords never meet each other, nor vertical ones, so g is the
// number of chords minus a maximum matching of the bipartite graph whose edges join a
// horizontal and a vertical chord that intersect (Konig's theorem).
//
// Pixel masks: pieces are the 4-connected components of the mask; holes are the
// 8-connected components of the background that do not touch the image border, each
// belonging to the piece that encloses it. A grid point where the mask occupies two
// diagonally opposite pixels of its 2 x 2 neighbourhood is split in two (a convex
// corner of each pixel), which is why the background is 8-connected.
#include <algorithm>
#include <cstring>
#include <queue>
#include <vector>

#include "common.cuh"

namespace devel {
namespace {

struct Chord {
    int line, a, b;  // horizontal: y, x from a to b; vertical: x, y from a to b
};

// Hopcroft-Karp maximum matching of a bipartite graph (adjacency of the left side)
int max_matching(int nl, int nr, const std::vector<std::vector<int>>& adj) {
    std::vector<int> ml(nl, -1), mr(nr, -1), dist(nl);
    int matched = 0;
    while (true) {
        std::queue<int> q;
        bool found = false;
        for (int u = 0; u < nl; ++u) {
            if (ml[u] < 0) {
                dist[u] = 0;
                q.push(u);
            } else {
                dist[u] = -1;
            }
        }
        while (!q.empty()) {
            const int u = q.front();
            q.pop();
            for (int v : adj[u]) {
                const int w = mr[v];
                if (w < 0) {
                    found = true;
                } else if (dist[w] < 0) {
                    dist[w] = dist[u] + 1;
                    q.push(w);
                }
            }
        }
        if (!found) break;
        // iterative DFS along the layered graph
        std::vector<size_t> it(nl, 0);
        for (int s = 0; s < nl; ++s) {
            if (ml[s] >= 0) continue;
            std::vector<int> stack{s};
            while (!stack.empty()) {
                const int u = stack.back();
                bool advanced = false;
                while (it[u] < adj[u].size()) {
                    const int v = adj[u][it[u]++];
                    const int w = mr[v];
                    if (w < 0) {
                        // augment along the stack
                        int vv = v;
                        for (int k = (int)stack.size() - 1; k >= 0; --k) {
                            const int uu = stack[k];
                            const int prev = ml[uu];
                            ml[uu] = vv;
                            mr[vv] = uu;
                            vv = prev;
                        }
                        ++matched;
                        stack.clear();
                        advanced = true;
                        break;
                    }
                    if (dist[w] == dist[u] + 1) {
                        stack.push_back(w);
                        advanced = true;
                        break;
                    }
                }
                if (!advanced) {
                    dist[u] = -1;  // dead end for this phase
                    stack.pop_back();
                }
            }
        }
    }
    return matched;
}

long long shot_count(int n, const unsigned char* mask) {
    const size_t N = (size_t)n * n;
    auto in = [&](int i, int j) { return i >= 0 && j >= 0 && i < n && j < n && mask[(size_t)i * n + j] != 0; };
    // pieces: 4-connected components of the mask
    std::vector<int> comp(N, -1);
    int ncomp = 0;
    std::vector<int> q;
    for (size_t p = 0; p < N; ++p) {
        if (!mask[p] || comp[p] >= 0) continue;
        q.assign(1, (int)p);
        comp[p] = ncomp;
        for (size_t h = 0; h < q.size(); ++h) {
            const int i = q[h] / n, j = q[h] % n;
            const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
            for (int d = 0; d < 4; ++d) {
                const int a = i + di[d], b = j + dj[d];
                if (in(a, b) && comp[(size_t)a * n + b] < 0) {
                    comp[(size_t)a * n + b] = ncomp;
                    q.push_back(a * n + b);
                }
            }
        }
        ++ncomp;
    }
    if (ncomp == 0) return 0;
    // holes: 8-connected background components away from the border, owned by the piece
    // holding the pixel above their first (row-major) pixel
    std::vector<long long> holes(ncomp, 0), verts(ncomp, 0);
    std::vector<char> seen(N, 0);
    for (size_t p = 0; p < N; ++p) {
        if (mask[p] || seen[p]) continue;
        q.assign(1, (int)p);
        seen[p] = 1;
        bool border = false;
        for (size_t h = 0; h < q.size(); ++h) {
            const int i = q[h] / n, j = q[h] % n;
            if (i == 0 || j == 0 || i == n - 1 || j == n - 1) border = true;
            for (int di = -1; di <= 1; ++di)
                for (int dj = -1; dj <= 1; ++dj) {
                    const int a = i + di, b = j + dj;
                    if (a < 0 || b < 0 || a >= n || b >= n) continue;
                    const size_t r = (size_t)a * n + b;
                    if (!mask[r] && !seen[r]) {
                        seen[r] = 1;
                        q.push_back((int)r);
                    }
                }
        }
        if (!border) {
            const int i = (int)(p / n), j = (int)(p % n);  // p is the first pixel in row-major order
            holes[comp[(size_t)(i - 1) * n + j]] += 1;
        }
    }
    // vertices: reflex (3 of 4 pixels), convex (1 of 4, or each side of a diagonal pair)
    // reflex direction codes: the missing quadrant 0 = top-left, 1 = top-right,
    // 2 = bottom-left, 3 = bottom-right (of the grid point)
    std::vector<signed char> reflex((size_t)(n + 1) * (n + 1), -1);
    auto at = [&](int i, int j) -> int { return in(i, j) ? comp[(size_t)i * n + j] : -1; };
    for (int i = 0; i <= n; ++i)
        for (int j = 0; j <= n; ++j) {
            const bool a = in(i - 1, j - 1), b = in(i - 1, j), c = in(i, j - 1), d = in(i, j);
            const int k = a + b + c + d;
            if (k == 1) {
                verts[a ? at(i - 1, j - 1) : b ? at(i - 1, j) : c ? at(i, j - 1) : at(i, j)] += 1;
            } else if (k == 3) {
                const int miss = !a ? 0 : !b ? 1 : !c ? 2 : 3;
                reflex[(size_t)i * (n + 1) + j] = (signed char)miss;
                verts[a ? at(i - 1, j - 1) : at(i - 1, j)] += 1;
            } else if (k == 2 && a == d) {  // diagonal pair: one convex corner on each side
                if (a) {
                    verts[at(i - 1, j - 1)] += 1;
                    verts[at(i, j)] += 1;
                } else {
                    verts[at(i - 1, j)] += 1;
                    verts[at(i, j - 1)] += 1;
                }
            }
        }
    // chords, each found from its left (top) end: a reflex vertex whose chord points
    // right (down) walks while both pixels along the segment are mask, and the chord
    // exists if the walk ends on a reflex vertex whose chord points back
    std::vector<std::vector<Chord>> hch(ncomp), vch(ncomp);
    for (int i = 0; i <= n; ++i)
        for (int j = 0; j <= n; ++j) {
            const int miss = reflex[(size_t)i * (n + 1) + j];
            if (miss < 0) continue;
            // horizontal chord direction: away from the missing quadrant's side
            const bool right = (miss == 0 || miss == 2), down = (miss == 0 || miss == 1);
            if (right) {
                int x = j;
                while (x < n && in(i - 1, x) && in(i, x)) ++x;
                if (x > j) {
                    const int m2 = reflex[(size_t)i * (n + 1) + x];
                    if (m2 == 1 || m2 == 3) hch[at(i, j)].push_back({i, j, x});
                }
            }
            if (down) {
                int y = i;
                while (y < n && in(y, j - 1) && in(y, j)) ++y;
                if (y > i) {
                    const int m2 = reflex[(size_t)y * (n + 1) + j];
                    if (m2 == 2 || m2 == 3) vch[at(i, j)].push_back({j, i, y});
                }
            }
        }
    long long total = 0;
    for (int c = 0; c < ncomp; ++c) {
        auto& H = hch[c];
        auto& V = vch[c];
        std::sort(V.begin(), V.end(), [](const Chord& p, const Chord& r) { return p.line < r.line; });
        std::vector<std::vector<int>> adj(H.size());
        for (size_t h = 0; h < H.size(); ++h) {
            auto lo = std::lower_bound(V.begin(), V.end(), H[h].a, [](const Chord& p, int x) { return p.line < x; });
            for (auto it = lo; it != V.end() && it->line <= H[h].b; ++it)
                if (H[h].line >= it->a && H[h].line <= it->b) adj[h].push_back((int)(it - V.begin()));
        }
        const long long g = (long long)H.size() + (long long)V.size() - max_matching((int)H.size(), (int)V.size(), adj);
        total += verts[c] / 2 + holes[c] - g - 1;
    }
    return total;
}

}  // namespace
}  // namespace devel

extern "C" int devel_shot_count(int n, const unsigned char* mask_host, long long* count_out) {
    using namespace devel;
    if (n < 1 || n > 16384) return set_error(DEVEL_EINVAL, "devel_shot_count: n=%d outside [1, 16384]", n);
    if (!mask_host || !count_out) return set_error(DEVEL_EINVAL, "devel_shot_count: NULL argument");
    *count_out = shot_count(n, mask_host);
    return DEVEL_OK;
}
