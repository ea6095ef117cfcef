/*
 * Polylla oracle -- TEST INFRASTRUCTURE, not part of the library.
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load this file's shared object.  The GPU library neither links
 * nor calls it, and it shares no header, helper or table with the CUDA code.
 *
 * A plain, slow, sequential restatement of the Polylla method of
 * "GPolylla: Fully GPU-accelerated polygonal mesh generator"
 * (Salinas-Fernandez, Carrasco, Hitschfeld-Kahler, arXiv 2403.14723):
 *
 *   Label phase      Algorithm 2 (longest edge), Algorithm 3 (frontier
 *                    edges), Algorithm 4 (seed edges)         -- Section 5.1
 *   Traversal phase  Algorithm 5                              -- Section 5.2
 *   Repair phase     Algorithm 6                              -- Section 5.3
 *   Output           every polygon listed from its smallest half-edge,
 *                    polygons in ascending order of that half-edge.
 *   Lepp             oracle_lepp: the longest-edge propagation path of
 *                    every triangle (Definition 1, Section 3.1) from the
 *                    longest edges of the label phase -- Section 1 lists
 *                    it as a reusable data-parallel building block.
 *
 * Half-edge queries follow Section 4 ("Half-edge representation" and its
 * CUDA subsection), with the garbled formulas read as:
 *   target(e)   = origin(twin(e))
 *   CW(e)       = next(twin(e))    rotation about origin(e), clockwise
 *   CCW(e)      = twin(prev(e))    rotation about origin(e), counter-clockwise
 *   degree(v)   = number of half-edges met rotating about v until the start
 *                 comes back
 *   edgeOfVertex(v) = the smallest interior half-edge whose origin is v
 * next/prev/twin/origin are read from the INPUT arrays (the paper's
 * mesh_input); the output links go to next_out/prev_out (mesh_output).
 *
 * Readings taken where the paper is silent, garbled or inconsistent:
 *  R1 squared lengths: d = dx*dx + dy*dy in IEEE binary64, round to nearest,
 *     each operation rounded on its own (compile with -ffp-contract=off);
 *     the longest edge is the largest d, ties going to the edge whose id
 *     min(e, twin e) is smaller (Algorithm 2 only says "max").
 *  R2 border edge: half-edge e or twin(e) lies in [3T, H) (the border
 *     half-edges appended after the triangles).
 *  R3 frontier (Algorithm 3, whose test names the wrong variable): e is a
 *     frontier edge iff it is a border edge or neither e nor twin(e) is a
 *     longest edge.
 *  R4 seeds (Algorithm 4 "label he or twin(he)"): the smaller half of a
 *     terminal edge; the interior half of a border terminal edge.
 *  R5 traversal (Algorithm 5, whose inner loop never advances): from the
 *     current frontier half-edge cur, x = next(cur), rotate x clockwise
 *     (CW) until it is a frontier edge, link cur -> x, continue from x,
 *     until the start comes back.  A polygon is non-simple when some cur
 *     gets next_out(cur) == twin(cur); target(cur) is then a barrier tip.
 *  R6 repair (Algorithm 6): the frontier half-edge f leaving a tip b and
 *     the rotation count are taken with the frontier labels of the label
 *     phase (F0); the loop "for 0 to (degree(b)-1)/2" is inclusive, so the
 *     middle edge is m = CW^r(f) with r = floor((d-1)/2) + 1.  Chords go to
 *     a second label array F1 = F0 + chords, which the repair traversals use.
 *  R7 completion: the paper presumes each terminal-edge region's boundary is
 *     reached from its seed.  After the seeds, every F0 frontier half-edge
 *     not yet visited starts one more traversal (counted in the statistics;
 *     zero on all meshes seen so far), so every frontier half-edge is linked.
 *  R8 output: polygons are the cycles of next_out over the F1 frontier
 *     interior half-edges, each listed from its smallest half-edge, sorted by
 *     that half-edge; v_list holds the origin of each listed half-edge.
 */
#define _POSIX_C_SOURCE 199309L
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

enum {
    OR_OK = 0,
    OR_ERR_ALLOC = -1,
    OR_ERR_NONTERMINATING = -2,
    OR_ERR_NOT_A_CYCLE = -3,
};

/* statistics slots */
enum {
    ST_SEEDS = 0,          /* seeds from Algorithm 4                        */
    ST_TIPS,               /* barrier tips repaired                          */
    ST_POLYGONS,           /* polygons in the output                         */
    ST_FRONTIER1,          /* F1 frontier interior half-edges (sum of lengths) */
    ST_NONSIMPLE,          /* non-simple polygons found by the traversal     */
    ST_COMPLETION,         /* traversals started by reading R7               */
    ST_REPAIR_POLYGONS,    /* polygons produced by repair traversals         */
    ST_TRAVERSAL_POLYGONS, /* polygons produced by the traversal phase       */
    ST_DISTINCT_CHORDS,    /* distinct chord edges                            */
    ST_FRONTIER0,          /* F0 frontier interior half-edges                 */
    ST_COUNT
};

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

typedef struct {
    int32_t V, T, H;
    const double *xy;
    const int32_t *origin, *twin, *next, *prev;
} mesh_t;

static int32_t q_target(const mesh_t *m, int32_t e) { return m->origin[m->twin[e]]; }
static int32_t q_cw(const mesh_t *m, int32_t e) { return m->next[m->twin[e]]; }
static int32_t q_ccw(const mesh_t *m, int32_t e) { return m->twin[m->prev[e]]; }
static int q_border_edge(const mesh_t *m, int32_t e) {
    int32_t hi = 3 * m->T;
    return e >= hi || m->twin[e] >= hi;
}

/* squared length of half-edge e, reading R1 */
static double sq_length(const mesh_t *m, int32_t e) {
    int32_t a = m->origin[e];
    int32_t b = q_target(m, e);
    double dx = m->xy[2 * (int64_t)b] - m->xy[2 * (int64_t)a];
    double dy = m->xy[2 * (int64_t)b + 1] - m->xy[2 * (int64_t)a + 1];
    double dx2 = dx * dx;
    double dy2 = dy * dy;
    return dx2 + dy2;
}

static int32_t edge_id(const mesh_t *m, int32_t e) {
    int32_t t = m->twin[e];
    return e < t ? e : t;
}

/* degree(v) by rotating about v from half-edge e (origin(e) == v) */
static int32_t degree_from(const mesh_t *m, int32_t e, int32_t cap) {
    int32_t d = 0, h = e;
    do {
        h = q_ccw(m, h);
        if (++d > cap) return -1;
    } while (h != e);
    return d;
}

/* Algorithm 5 under frontier labels F, from half-edge s.  Writes next_out
 * and prev_out, marks visited half-edges, appends the polygon's half-edges
 * to poly (if non-NULL) and the half-edges entering a barrier tip to tips.
 * Returns the polygon length, or a negative status. */
static int64_t traverse(const mesh_t *m, const uint8_t *F, int32_t s,
                        int32_t *next_out, int32_t *prev_out, uint8_t *visited,
                        int32_t *poly, int32_t *tips, int32_t *n_tips) {
    int64_t cap = (int64_t)m->H + 1;
    int32_t h = s;
    int64_t guard = 0;
    while (!F[h]) {
        h = q_cw(m, h);
        if (++guard > cap) return OR_ERR_NONTERMINATING;
    }
    int32_t init = h, cur = init;
    int64_t len = 0;
    do {
        int32_t x = m->next[cur];
        guard = 0;
        while (!F[x]) {
            x = q_cw(m, x);
            if (++guard > cap) return OR_ERR_NONTERMINATING;
        }
        next_out[cur] = x;
        prev_out[x] = cur;
        if (visited) visited[cur] = 1;
        if (poly) poly[len] = cur;
        if (tips && x == m->twin[cur]) tips[(*n_tips)++] = cur;
        len++;
        if (len > cap) return OR_ERR_NONTERMINATING;
        cur = x;
    } while (cur != init);
    return len;
}

int oracle_stats_count(void) { return ST_COUNT; }

/*
 * Run the whole method.  Array capacities: longest/frontier0/frontier1,
 * next_out/prev_out [H]; seed_list [H]; tip_in/chord [V]; seeds [T];
 * offsets [T+1]; he_list/v_list [3T].  stats [ST_COUNT]; times [6] seconds
 * (longest edge, frontier, seeds, traversal, repair, output).
 */
int oracle_polylla(int32_t V, int32_t T, int32_t H, const double *coords,
                   const int32_t *origin, const int32_t *twin,
                   const int32_t *next, const int32_t *prev,
                   uint8_t *longest, uint8_t *frontier0, uint8_t *frontier1,
                   int32_t *seed_list, int32_t *tip_in, int32_t *chord,
                   int32_t *next_out, int32_t *prev_out,
                   int32_t *seeds, int32_t *offsets, int32_t *he_list, int32_t *v_list,
                   int64_t *stats, double *times) {
    mesh_t M = {V, T, H, coords, origin, twin, next, prev};
    const mesh_t *m = &M;
    const int32_t HI = 3 * T;
    int status = OR_OK;
    for (int i = 0; i < ST_COUNT; i++) stats[i] = 0;
    for (int i = 0; i < 6; i++) times[i] = 0.0;

    uint8_t *visited = (uint8_t *)calloc((size_t)H, 1);
    uint8_t *usage = (uint8_t *)calloc((size_t)H, 1);
    int32_t *poly = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H + 1));
    int32_t *edge_of_vertex = (int32_t *)malloc(sizeof(int32_t) * (size_t)(V > 0 ? V : 1));
    /* tips found by the traversal phase, grouped per non-simple polygon:
     * polygon p owns tips_all[tips_start[p] .. tips_start[p+1]) */
    int32_t *tips_all = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H + 1));
    int64_t *tips_start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(H + 2));
    int32_t *subseeds = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * (int64_t)H + 2));
    if (!visited || !usage || !poly || !edge_of_vertex || !tips_all || !tips_start || !subseeds) {
        status = OR_ERR_ALLOC;
        goto done;
    }

    /* ---- Algorithm 2: longest edge of each triangle ---------------------- */
    double t0 = now_s();
    memset(longest, 0, (size_t)H);
    for (int32_t t = 0; t < T; t++) {
        int32_t he = 3 * t;                 /* incidentHalfedge(t) */
        int32_t cand[3] = {he, m->next[he], m->prev[he]};
        int32_t best = cand[0];
        double dbest = sq_length(m, best);
        for (int k = 1; k < 3; k++) {
            double d = sq_length(m, cand[k]);
            if (d > dbest || (d == dbest && edge_id(m, cand[k]) < edge_id(m, best))) {
                best = cand[k];
                dbest = d;
            }
        }
        longest[best] = 1;
    }
    double t1 = now_s();
    times[0] = t1 - t0;

    /* ---- Algorithm 3: frontier edges (reading R3) ----------------------- */
    for (int32_t e = 0; e < H; e++) {
        frontier0[e] = (uint8_t)(q_border_edge(m, e) || (!longest[e] && !longest[m->twin[e]]));
    }
    double t2 = now_s();
    times[1] = t2 - t1;

    /* ---- Algorithm 4: seed edges (reading R4) --------------------------- */
    int32_t n_seeds = 0;
    for (int32_t e = 0; e < H; e++) {
        int32_t tw = m->twin[e];
        int border = q_border_edge(m, e);
        int terminal = longest[e] && longest[tw] && !border;
        int border_terminal = border && (longest[e] || longest[tw]);
        if (terminal && e < tw) seed_list[n_seeds++] = e;
        else if (border_terminal && e < HI) seed_list[n_seeds++] = e;
    }
    stats[ST_SEEDS] = n_seeds;
    double t3 = now_s();
    times[2] = t3 - t2;

    /* ---- Algorithm 5: traversal from every seed, then reading R7 -------- */
    memcpy(next_out, next, sizeof(int32_t) * (size_t)H);
    memcpy(prev_out, prev, sizeof(int32_t) * (size_t)H);
    int64_t n_nonsimple = 0, n_trav_polys = 0, n_completion = 0;
    int32_t n_tips_found = 0;
    int32_t scan = 0;
    tips_start[0] = 0;
    for (int64_t i = 0;; i++) {
        int32_t s;
        if (i < n_seeds) {
            s = seed_list[i];
        } else {
            /* reading R7: frontier interior half-edges no seed reached */
            while (scan < HI && !(frontier0[scan] && !visited[scan])) scan++;
            if (scan >= HI) break;
            s = scan;
            n_completion++;
        }
        int32_t nt = 0;
        int64_t len = traverse(m, frontier0, s, next_out, prev_out, visited, NULL,
                               tips_all + n_tips_found, &nt);
        if (len < 0) { status = (int)len; goto done; }
        n_trav_polys++;
        if (nt > 0) {
            n_tips_found += nt;
            n_nonsimple++;
            tips_start[n_nonsimple] = n_tips_found;
        }
    }
    stats[ST_NONSIMPLE] = n_nonsimple;
    stats[ST_COMPLETION] = n_completion;
    double t4 = now_s();
    times[3] = t4 - t3;

    /* ---- Algorithm 6: repair every non-simple polygon ------------------- */
    memcpy(frontier1, frontier0, (size_t)H);
    for (int32_t v = 0; v < V; v++) edge_of_vertex[v] = -1;
    for (int32_t e = HI - 1; e >= 0; e--) edge_of_vertex[m->origin[e]] = e;
    int32_t n_tips_total = 0;
    int64_t n_repair_polys = 0;
    for (int64_t p = 0; p < n_nonsimple; p++) {
        int32_t n_sub = 0;
        for (int64_t q = tips_start[p]; q < tips_start[p + 1]; q++) {
            int32_t cin = tips_all[q];          /* half-edge entering the tip */
            int32_t b = q_target(m, cin);
            int32_t e = edge_of_vertex[b];
            int64_t guard = 0;
            while (!frontier0[e]) {
                e = q_cw(m, e);
                if (++guard > H) { status = OR_ERR_NONTERMINATING; goto done; }
            }
            int32_t f = e;
            int32_t d = degree_from(m, f, H);
            if (d < 0) { status = OR_ERR_NONTERMINATING; goto done; }
            for (int32_t r = 0; r <= (d - 1) / 2; r++) e = q_cw(m, e);
            int32_t tw = m->twin[e];
            tip_in[n_tips_total] = f;
            chord[n_tips_total] = e;
            n_tips_total++;
            frontier1[e] = 1;
            frontier1[tw] = 1;
            subseeds[n_sub++] = e;
            subseeds[n_sub++] = tw;
            usage[e] = 1;
            usage[tw] = 1;
        }
        for (int32_t k = 0; k < n_sub; k++) {
            int32_t h = subseeds[k];
            if (!usage[h]) continue;
            usage[h] = 0;
            int64_t l2 = traverse(m, frontier1, h, next_out, prev_out, visited, poly, NULL, NULL);
            if (l2 < 0) { status = (int)l2; goto done; }
            for (int64_t q = 0; q < l2; q++) usage[poly[q]] = 0;
            n_repair_polys++;
        }
    }
    stats[ST_TIPS] = n_tips_total;
    stats[ST_REPAIR_POLYGONS] = n_repair_polys;
    stats[ST_TRAVERSAL_POLYGONS] = n_trav_polys - n_nonsimple;
    {
        /* distinct chord edges, counted once per undirected edge */
        uint8_t *seen = (uint8_t *)calloc((size_t)H, 1);
        if (!seen) { status = OR_ERR_ALLOC; goto done; }
        int64_t distinct = 0;
        for (int32_t k = 0; k < n_tips_total; k++) {
            int32_t id = edge_id(m, chord[k]);
            if (!seen[id]) { seen[id] = 1; distinct++; }
        }
        free(seen);
        stats[ST_DISTINCT_CHORDS] = distinct;
    }
    double t5 = now_s();
    times[4] = t5 - t4;

    /* ---- output: cycles of next_out, canonical order (reading R8) ------- */
    memset(visited, 0, (size_t)H);
    int64_t n_poly = 0, k = 0, n_f0 = 0, n_f1 = 0;
    for (int32_t e = 0; e < HI; e++) {
        n_f0 += frontier0[e];
        n_f1 += frontier1[e];
    }
    for (int32_t e = 0; e < HI; e++) {
        if (!frontier1[e] || visited[e]) continue;
        seeds[n_poly] = e;
        offsets[n_poly] = (int32_t)k;
        int32_t cur = e;
        int64_t len = 0;
        do {
            if (cur < 0 || cur >= HI || !frontier1[cur] || visited[cur]) {
                status = OR_ERR_NOT_A_CYCLE;
                goto done;
            }
            visited[cur] = 1;
            he_list[k] = cur;
            v_list[k] = m->origin[cur];
            k++;
            len++;
            cur = next_out[cur];
        } while (cur != e);
        n_poly++;
    }
    offsets[n_poly] = (int32_t)k;
    stats[ST_POLYGONS] = n_poly;
    stats[ST_FRONTIER1] = k;
    stats[ST_FRONTIER0] = n_f0;
    if (k != n_f1) status = OR_ERR_NOT_A_CYCLE;
    times[5] = now_s() - t5;

done:
    free(visited);
    free(usage);
    free(poly);
    free(edge_of_vertex);
    free(tips_all);
    free(tips_start);
    free(subseeds);
    return status;
}

/*
 * Lepp (Definition 1): Lepp(t0) is t0, t1, ..., where t_i is the neighbour
 * of t_{i-1} across the longest edge of t_{i-1}; it ends at the terminal
 * edge, the longest edge shared by the last two triangles (both have it as
 * their longest edge), or at a longest edge on the border.  Reading (the
 * definition's indices are garbled): the path lists every triangle met,
 * the last two triangles of an interior terminal edge included, so its
 * length is 1 for a triangle whose longest edge is a border edge.
 *
 * For every triangle t: terminal[t] = the seed half-edge of the terminal
 * edge (reading R4: the smaller half of an interior terminal edge, the
 * interior half of a border one), length[t] = number of triangles in
 * Lepp(t).  longest[H] is the label phase's longest-edge flag per
 * half-edge.  Returns OR_OK, or OR_ERR_NONTERMINATING when a path exceeds T
 * triangles (impossible under reading R1's strict order).
 */
int oracle_lepp(int32_t T, int32_t H, const int32_t *twin, const uint8_t *longest,
                int32_t *terminal, int32_t *length) {
    const int32_t HI = 3 * T;
    (void)H;
    for (int32_t t0 = 0; t0 < T; t0++) {
        int32_t t = t0, n = 1;
        for (;;) {
            int32_t e = 3 * t;               /* the longest half-edge of t */
            while (!longest[e]) e++;
            const int32_t tw = twin[e];
            if (tw >= HI) {                  /* border: e is a border-terminal edge */
                terminal[t0] = e;
                break;
            }
            const int32_t t1 = tw / 3;       /* the neighbour across it */
            n++;
            if (longest[tw]) {               /* shared longest edge: terminal */
                terminal[t0] = e < tw ? e : tw;
                break;
            }
            t = t1;
            if (n > T + 1) return OR_ERR_NONTERMINATING;
        }
        length[t0] = n;
    }
    return OR_OK;
}

/* The path itself: the triangles of Lepp(t0) in order into path (capacity
 * cap); returns its length, or -1 when cap is too small. */
int32_t oracle_lepp_path(int32_t T, const int32_t *twin, const uint8_t *longest, int32_t t0,
                         int32_t *path, int32_t cap) {
    const int32_t HI = 3 * T;
    int32_t t = t0, n = 0;
    if (n >= cap) return -1;
    path[n++] = t;
    for (;;) {
        int32_t e = 3 * t;
        while (!longest[e]) e++;
        const int32_t tw = twin[e];
        if (tw >= HI) return n;
        if (n >= cap) return -1;
        path[n++] = tw / 3;
        if (longest[tw]) return n;
        t = tw / 3;
    }
}

/*
 * Convexification (post-processing).  Section 4.2 notes that keeping every
 * half-edge of the triangulation (relinking instead of deleting) allows a
 * later step to turn non-convex polygons into convex ones; the paper gives
 * no method.  Reading R9, with only orientation tests:
 *   - a corner of a polygon is a frontier half-edge e with x = next_out[e];
 *     it sits at v = target(e).  Directions leave v: dir(h) = target(h) - v
 *     for a half-edge h leaving v; the corner's first side is twin(e), so
 *     dir(twin e) = origin(e) - v.
 *   - cross(a, b) = a.x * b.y - a.y * b.x, each operation in IEEE binary64
 *     rounded on its own.  b lies within a half turn clockwise of a iff
 *     cross(a, b) <= 0.
 *   - the corner is reflex iff x is not within a half turn clockwise of
 *     twin(e): cross(dir(twin e), dir(x)) > 0.
 *   - the candidates of a corner are the half-edges leaving v strictly
 *     inside it, in clockwise order: y_1 = next(e) (the triangle's), then
 *     y_{i+1} = CW(y_i), up to (not including) x -- the rotation of the
 *     traversal, over the non-frontier half-edges it skipped.
 *   - at a reflex corner, from cur = twin(e): take the last candidate after
 *     cur that lies within a half turn clockwise of cur, make it a chord and
 *     continue from it, until x lies within a half turn of cur.  (Farthest
 *     first: the fewest chords that leave every part of the corner at most
 *     a half turn.)
 *   - F2 = F1 plus both halves of every chord; the polygons are the
 *     traversal (reading R5) under F2, listed as in reading R8.
 * Corners are processed independently from F1 and next_out, so the result
 * does not depend on their order.  A corner left reflex because its
 * candidates ran out (not possible when every triangle has positive area)
 * is counted in stats[3].
 *
 * In:  the mesh's input arrays; frontier1 [H] and next_out [H] of
 *      oracle_polylla.
 * Out: frontier2 [H]; next2, prev2 [H]; chords [3T] (the chosen half-edges,
 *      each leaving its corner's vertex; *n_chords of them); the CSR seeds
 *      [T], offsets [T+1], he_list, v_list [3T]; stats[0] polygons,
 *      stats[1] F2 frontier interior half-edges, stats[2] reflex corners,
 *      stats[3] corners left reflex, stats[4] distinct chord edges.
 */
static void half_dir(const mesh_t *m, int32_t h, int32_t v, double *dx, double *dy) {
    /* direction of the half-edge h leaving v: target(h) - v */
    const int32_t t = q_target(m, h);
    *dx = m->xy[2 * (int64_t)t] - m->xy[2 * (int64_t)v];
    *dy = m->xy[2 * (int64_t)t + 1] - m->xy[2 * (int64_t)v + 1];
}

static double cross2(double ax, double ay, double bx, double by) {
    const double p = ax * by;
    const double q = ay * bx;
    return p - q;
}

int oracle_convexify(int32_t V, int32_t T, int32_t H, const double *coords,
                     const int32_t *origin, const int32_t *twin, const int32_t *next, const int32_t *prev,
                     const uint8_t *frontier1, const int32_t *next_out,
                     uint8_t *frontier2, int32_t *next2, int32_t *prev2,
                     int32_t *chords, int32_t *n_chords,
                     int32_t *seeds, int32_t *offsets, int32_t *he_list, int32_t *v_list,
                     int64_t *stats) {
    mesh_t mesh = {V, T, H, coords, origin, twin, next, prev};
    const mesh_t *m = &mesh;
    const int32_t HI = 3 * T;
    int status = OR_OK;
    int64_t n_reflex = 0, n_left = 0;
    int32_t nc = 0;
    uint8_t *visited = (uint8_t *)calloc((size_t)H, 1);
    int32_t *fan = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H + 1));
    if (!visited || !fan) { status = OR_ERR_ALLOC; goto done; }
    memcpy(frontier2, frontier1, (size_t)H);

    /* ---- chords at reflex corners ---- */
    for (int32_t e = 0; e < HI; e++) {
        if (!frontier1[e]) continue;
        const int32_t x = next_out[e];
        const int32_t v = q_target(m, e);
        double ux, uy, wx, wy;
        half_dir(m, twin[e], v, &ux, &uy);
        half_dir(m, x, v, &wx, &wy);
        if (!(cross2(ux, uy, wx, wy) > 0.0)) continue;
        n_reflex++;
        /* the candidates, clockwise from the triangle's next half-edge */
        int32_t n_fan = 0, y = next[e];
        while (y != x) {
            if (n_fan > H) { status = OR_ERR_NONTERMINATING; goto done; }
            fan[n_fan++] = y;
            y = q_cw(m, y);
        }
        int32_t i = 0;                       /* next candidate after cur */
        while (cross2(ux, uy, wx, wy) > 0.0) {
            int32_t best = -1;
            while (i < n_fan) {
                double dx, dy;
                half_dir(m, fan[i], v, &dx, &dy);
                if (cross2(ux, uy, dx, dy) <= 0.0) {
                    best = i;
                    i++;
                } else {
                    break;
                }
            }
            if (best < 0) {                  /* no candidate within a half turn */
                n_left++;
                break;
            }
            const int32_t c = fan[best];
            frontier2[c] = 1;
            frontier2[twin[c]] = 1;
            chords[nc++] = c;
            half_dir(m, c, v, &ux, &uy);
        }
    }
    *n_chords = nc;

    /* ---- relink under F2 (reading R5), every frontier half-edge ---- */
    memcpy(next2, next, sizeof(int32_t) * (size_t)H);
    memcpy(prev2, prev, sizeof(int32_t) * (size_t)H);
    for (int32_t e = 0; e < HI; e++) {
        if (!frontier2[e] || visited[e]) continue;
        const int64_t len = traverse(m, frontier2, e, next2, prev2, visited, NULL, NULL, NULL);
        if (len < 0) { status = (int)len; goto done; }
    }

    /* ---- output (reading R8) ---- */
    memset(visited, 0, (size_t)H);
    int64_t n_poly = 0, k = 0;
    for (int32_t e = 0; e < HI; e++) {
        if (!frontier2[e] || visited[e]) continue;
        seeds[n_poly] = e;
        offsets[n_poly] = (int32_t)k;
        int32_t cur = e;
        do {
            if (cur < 0 || cur >= HI || !frontier2[cur] || visited[cur]) {
                status = OR_ERR_NOT_A_CYCLE;
                goto done;
            }
            visited[cur] = 1;
            he_list[k] = cur;
            v_list[k] = origin[cur];
            k++;
            cur = next2[cur];
        } while (cur != e);
        n_poly++;
    }
    offsets[n_poly] = (int32_t)k;
    {
        /* distinct chord edges */
        int64_t distinct = 0;
        memset(visited, 0, (size_t)H);
        for (int32_t j = 0; j < nc; j++) {
            const int32_t id = edge_id(m, chords[j]);
            if (!visited[id]) { visited[id] = 1; distinct++; }
        }
        stats[4] = distinct;
    }
    stats[0] = n_poly;
    stats[1] = k;
    stats[2] = n_reflex;
    stats[3] = n_left;

done:
    free(visited);
    free(fan);
    return status;
}
