/*
 * fem_oracle.c -- plain, single-threaded CPU oracle for frequent-episode counting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or constant with the CUDA
 * library, and it does not read the CUDA library's outputs.
 *
 * What it computes (Cao et al., "Towards Chip-on-Chip Neuroscience: Fast Mining
 * of Frequent Episodes Using Graphics Processors"):
 *   - an event stream is a time-ordered list of (type, time) pairs (Def. 2.1);
 *   - a serial episode is an ordered tuple of N event types (Def. 2.2) with one
 *     inter-event interval (lo, hi] per edge (Section 2, temporal constraints);
 *   - its frequency is the size of the largest set of non-overlapped
 *     occurrences (Section 2, frequency of episodes).
 *
 * Index conventions: the paper numbers episode nodes 1..N; this file uses
 * 0..N-1.  Edge k (0 <= k < N-1) joins node k to node k+1 with interval
 * (lo[k], hi[k]].  Times are unsigned 32-bit microseconds; every subtraction
 * below is (later time) - (earlier time) and cannot wrap because the stream is
 * time-sorted.
 *
 * Readings of the paper used here (each is listed with its reason in the
 * design notes of the repository):
 *   R1  Algorithm 1 tests the completing node with "i = |alpha| - 1"; the only
 *       consistent reading (and the one Algorithm 3 prints) is i = |alpha|.
 *   R2  Algorithm 3 checks only t - s <= hi (no positive lower bound), so the
 *       relaxed pass admits zero delays; the exact pass keeps lo < t - t'
 *       strictly, so two events with equal times never chain in it.
 *   R3  A one-node episode completes on every event of its type.
 *   R4  An unset slot in Algorithm 3 never satisfies the check.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LMAX 8

enum { ORC_RELAXED = 0, ORC_EXACT = 1, ORC_EXACT_LISTS = 2 };

/* ------------------------------------------------------------------------ */
/* A growable list of timestamps with a movable front (used as the list s[k]). */
typedef struct {
    uint32_t *v;
    int64_t head, len, cap; /* live entries are v[head .. len) */
} tlist;

static int tl_push(tlist *l, uint32_t x)
{
    if (l->len == l->cap) {
        /* compact first, then grow */
        if (l->head > 0) {
            memmove(l->v, l->v + l->head, (size_t)(l->len - l->head) * sizeof(uint32_t));
            l->len -= l->head;
            l->head = 0;
        }
        if (l->len == l->cap) {
            int64_t nc = l->cap ? 2 * l->cap : 16;
            uint32_t *nv = (uint32_t *)realloc(l->v, (size_t)nc * sizeof(uint32_t));
            if (!nv) return -1;
            l->v = nv;
            l->cap = nc;
        }
    }
    l->v[l->len++] = x;
    return 0;
}

static void tl_clear(tlist *l) { l->head = l->len = 0; }
static void tl_free(tlist *l) { free(l->v); l->v = NULL; l->head = l->len = l->cap = 0; }

/* ------------------------------------------------------------------------ */
/*
 * Algorithm 1 (Section 5.1), written as printed apart from reading R1: for
 * every event, walk the episode's nodes from last to first; on a type match
 * at node i > 0 scan s[i-1] from newest to oldest for a time t' with
 * lo < t - t' <= hi; on success either complete an occurrence (i = N-1:
 * count it, empty every list, stop handling this event) or append t to s[i].
 * Node 0 appends t to s[0] unconditionally.  Lists are never pruned.
 * Returns the count, or UINT32_MAX if memory ran out.
 */
uint32_t orc_count_exact_lists(const uint8_t *type, const uint32_t *t, int64_t n,
                               int N, const uint8_t *E, const uint32_t *lo,
                               const uint32_t *hi)
{
    uint32_t count = 0;
    tlist s[ORC_LMAX];
    memset(s, 0, sizeof(s));
    for (int64_t j = 0; j < n; j++) {
        for (int i = N - 1; i >= 0; i--) {
            if (type[j] != E[i]) continue;
            if (i == 0) {
                if (N == 1) { count++; break; }                 /* R3 */
                if (tl_push(&s[0], t[j])) goto oom;
                continue;
            }
            int found = 0;
            for (int64_t k = s[i - 1].len - 1; k >= s[i - 1].head; k--) {
                uint32_t d = t[j] - s[i - 1].v[k];
                if (lo[i - 1] < d && d <= hi[i - 1]) { found = 1; break; }
            }
            if (!found) continue;
            if (i == N - 1) {                                    /* R1 */
                count++;
                for (int k = 0; k < N; k++) tl_clear(&s[k]);
                break;                                           /* next event */
            }
            if (tl_push(&s[i], t[j])) goto oom;
        }
    }
    for (int k = 0; k < ORC_LMAX; k++) tl_free(&s[k]);
    return count;
oom:
    for (int k = 0; k < ORC_LMAX; k++) tl_free(&s[k]);
    return UINT32_MAX;
}

/* ------------------------------------------------------------------------ */
/*
 * One step of the exact machine with pruned lists (the windowed reading of
 * Algorithm 1).  Because times never decrease, an entry t' of s[k] with
 * t - t' > hi[k] can never satisfy edge k again; dropping it changes no
 * result.  After dropping such entries from the front, every remaining entry
 * satisfies t - t' <= hi[k], and the oldest one has the largest delay, so a
 * match exists iff the list is non-empty and t - front > lo[k].
 * Returns 1 if the event completed an occurrence (the lists are then empty).
 */
static int exact_step(tlist *s, int N, const uint8_t *E, const uint32_t *lo,
                      const uint32_t *hi, uint8_t ty, uint32_t tt, int *oom)
{
    for (int i = N - 1; i >= 0; i--) {
        if (ty != E[i]) continue;
        if (i == 0) {
            if (N == 1) return 1;                                /* R3 */
            tlist *L = &s[0];
            while (L->head < L->len && tt - L->v[L->head] > hi[0]) L->head++;
            if (tl_push(L, tt)) { *oom = 1; return 0; }
            continue;
        }
        tlist *P = &s[i - 1];
        while (P->head < P->len && tt - P->v[P->head] > hi[i - 1]) P->head++;
        if (!(P->head < P->len && tt - P->v[P->head] > lo[i - 1])) continue;
        if (i == N - 1) {
            for (int k = 0; k < N; k++) tl_clear(&s[k]);
            return 1;
        }
        tlist *L = &s[i];
        while (L->head < L->len && tt - L->v[L->head] > hi[i]) L->head++;
        if (tl_push(L, tt)) { *oom = 1; return 0; }
    }
    return 0;
}

/*
 * One step of Algorithm 3 (Section 5.3.1): one slot per node, holding the
 * latest time admitted at that node (Observation 5.1).  Node i > 0 admits t
 * if slot i-1 is set and t - s[i-1] <= hi[i-1] (readings R2, R4).
 * Returns 1 if the event completed an occurrence (every slot is then unset).
 */
static int relaxed_step(uint32_t *s, uint8_t *set, int N, const uint8_t *E,
                        const uint32_t *hi, uint8_t ty, uint32_t tt)
{
    for (int i = N - 1; i >= 0; i--) {
        if (ty != E[i]) continue;
        if (i == 0) {
            if (N == 1) return 1;                                /* R3 */
            s[0] = tt;
            set[0] = 1;
            continue;
        }
        if (!(set[i - 1] && tt - s[i - 1] <= hi[i - 1])) continue;
        if (i == N - 1) {
            memset(set, 0, (size_t)N);
            return 1;
        }
        s[i] = tt;
        set[i] = 1;
    }
    return 0;
}

/* Algorithm 1 with pruned lists over the whole stream. */
uint32_t orc_count_exact(const uint8_t *type, const uint32_t *t, int64_t n, int N,
                         const uint8_t *E, const uint32_t *lo, const uint32_t *hi)
{
    tlist s[ORC_LMAX];
    memset(s, 0, sizeof(s));
    uint32_t count = 0;
    int oom = 0;
    for (int64_t j = 0; j < n && !oom; j++)
        count += (uint32_t)exact_step(s, N, E, lo, hi, type[j], t[j], &oom);
    for (int k = 0; k < ORC_LMAX; k++) tl_free(&s[k]);
    return oom ? UINT32_MAX : count;
}

/* Algorithm 3 over the whole stream. */
uint32_t orc_count_relaxed(const uint8_t *type, const uint32_t *t, int64_t n, int N,
                           const uint8_t *E, const uint32_t *hi)
{
    uint32_t s[ORC_LMAX];
    uint8_t set[ORC_LMAX];
    memset(set, 0, sizeof(set));
    uint32_t count = 0;
    for (int64_t j = 0; j < n; j++)
        count += (uint32_t)relaxed_step(s, set, N, E, hi, type[j], t[j]);
    return count;
}

/*
 * Count m candidates, one after the other (the per-episode loop that the
 * per-thread-per-episode mapping of Section 5.2.1 parallelises).
 * Candidate c has len[c] nodes types[c*8 ..], edge intervals lo/hi[c*7 ..].
 * pass: ORC_RELAXED (Algorithm 3), ORC_EXACT (Algorithm 1, pruned lists) or
 * ORC_EXACT_LISTS (Algorithm 1, unpruned lists).
 */
int orc_count_batch(const uint8_t *type, const uint32_t *t, int64_t n, int64_t m,
                    const uint8_t *len, const uint8_t *types, const uint32_t *lo,
                    const uint32_t *hi, int pass, uint32_t *out)
{
    for (int64_t c = 0; c < m; c++) {
        int N = len[c];
        if (N < 1 || N > ORC_LMAX) return -1;
        const uint8_t *E = types + c * ORC_LMAX;
        const uint32_t *L = lo + c * (ORC_LMAX - 1);
        const uint32_t *H = hi + c * (ORC_LMAX - 1);
        if (pass == ORC_RELAXED)
            out[c] = orc_count_relaxed(type, t, n, N, E, H);
        else if (pass == ORC_EXACT)
            out[c] = orc_count_exact(type, t, n, N, E, L, H);
        else if (pass == ORC_EXACT_LISTS)
            out[c] = orc_count_exact_lists(type, t, n, N, E, L, H);
        else
            return -1;
        if (out[c] == UINT32_MAX) return -2;
    }
    return 0;
}

/*
 * Algorithm 4 (Section 5.3.2): relaxed count of every candidate, drop those
 * whose relaxed count is below theta, exact count of the rest.  survived[c] is
 * 1 for kept candidates; exact[c] is 0 for dropped ones.
 */
int orc_two_pass(const uint8_t *type, const uint32_t *t, int64_t n, int64_t m,
                 const uint8_t *len, const uint8_t *types, const uint32_t *lo,
                 const uint32_t *hi, uint32_t theta, uint32_t *relaxed,
                 uint32_t *exact, uint8_t *survived)
{
    int rc = orc_count_batch(type, t, n, m, len, types, lo, hi, ORC_RELAXED, relaxed);
    if (rc) return rc;
    for (int64_t c = 0; c < m; c++) {
        survived[c] = relaxed[c] >= theta;
        exact[c] = 0;
        if (!survived[c]) continue;
        int N = len[c];
        exact[c] = orc_count_exact(type, t, n, N, types + c * ORC_LMAX,
                                   lo + c * (ORC_LMAX - 1), hi + c * (ORC_LMAX - 1));
        if (exact[c] == UINT32_MAX) return -2;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/*
 * MapConcatenate (Section 5.2.2), in an exact form with entry classes.
 *
 * The stream is cut into P index ranges [b[p], b[p+1]).  W = sum of hi over
 * the episode's edges bounds the time span of any occurrence.  The serial
 * machine's behaviour from the start L of a segment on depends only on its
 * last completion r before L: if r is earlier than the first event w with
 * t >= t[L] - W (class "none"), the machine acts exactly like a fresh machine
 * started at w; otherwise it acts like a fresh machine started at r + 1, and
 * r is one of the last-node events in [w, L).  The Map step tabulates, for
 * every class, the completions inside the segment and the class handed to
 * the next segment; the Concatenate step composes the tables left to right
 * starting from class "none" (matching classes by event index, never by time).
 */
#define ORC_NONE (-1)

typedef struct {
    int64_t cls;      /* ORC_NONE or an event index */
    uint32_t count;   /* completions at indices in [L, R) */
    int64_t exit;     /* class handed to the next segment */
} orc_entry;

/* Run a fresh machine over [from, R); count completions at index >= L; return
 * the last completion index in *last (ORC_NONE if there was none). */
static int run_machine(const uint8_t *type, const uint32_t *t, int64_t from, int64_t L,
                       int64_t R, int N, const uint8_t *E, const uint32_t *lo,
                       const uint32_t *hi, int pass, uint32_t *count, int64_t *last)
{
    tlist s[ORC_LMAX];
    uint32_t slot[ORC_LMAX];
    uint8_t set[ORC_LMAX];
    memset(s, 0, sizeof(s));
    memset(set, 0, sizeof(set));
    int oom = 0;
    *count = 0;
    *last = ORC_NONE;
    for (int64_t j = from; j < R; j++) {
        int done = pass == ORC_RELAXED
                       ? relaxed_step(slot, set, N, E, hi, type[j], t[j])
                       : exact_step(s, N, E, lo, hi, type[j], t[j], &oom);
        if (oom) break;
        if (done) {
            *last = j;
            if (j >= L) (*count)++;
        }
    }
    for (int k = 0; k < ORC_LMAX; k++) tl_free(&s[k]);
    return oom ? -2 : 0;
}

/* First index j in [0, L] with t[j] >= t[L] - W (0 if t[L] < W). */
static int64_t window_start(const uint32_t *t, int64_t L, uint64_t W)
{
    if ((uint64_t)t[L] < W) return 0;
    uint32_t x = (uint32_t)((uint64_t)t[L] - W);
    int64_t j = L;
    while (j > 0 && t[j - 1] >= x) j--;
    return j;
}

/*
 * Exact MapConcatenate count of one episode over the segmentation b[0..P]
 * (b[0] = 0, b[P] = n, strictly increasing).  Returns the composed count, or
 * UINT32_MAX on error.  If tables_out is not NULL, the number of table
 * entries of segment p is written to tables_out[p] (a size check for tests).
 */
uint32_t orc_count_mapconcat(const uint8_t *type, const uint32_t *t, int64_t n, int N,
                             const uint8_t *E, const uint32_t *lo, const uint32_t *hi,
                             int pass, int64_t P, const int64_t *b, int64_t *tables_out)
{
    if (P < 1 || b[0] != 0 || b[P] != n) return UINT32_MAX;
    uint64_t W = 0;
    for (int k = 0; k + 1 < N; k++) W += hi[k];
    int64_t cls = ORC_NONE;   /* class entering the current segment */
    uint32_t total = 0;
    for (int64_t p = 0; p < P; p++) {
        int64_t L = b[p], R = b[p + 1];
        if (R <= L) return UINT32_MAX;
        int64_t w = window_start(t, L, W);
        int64_t wn = R < n ? window_start(t, R, W) : R;
        /* Map: one table entry for "none" and one per last-node event in [w, L). */
        int64_t nent = 1;
        for (int64_t j = w; j < L; j++) nent += type[j] == E[N - 1];
        orc_entry *tab = (orc_entry *)malloc((size_t)nent * sizeof(orc_entry));
        if (!tab) return UINT32_MAX;
        int64_t e = 0;
        for (int64_t j = w - 1; j < L; j++) {
            int64_t c;
            if (j == w - 1) c = ORC_NONE;
            else if (type[j] == E[N - 1]) c = j;
            else continue;
            uint32_t cnt;
            int64_t last;
            int64_t from = c == ORC_NONE ? w : c + 1;
            if (run_machine(type, t, from, L, R, N, E, lo, hi, pass, &cnt, &last)) {
                free(tab);
                return UINT32_MAX;
            }
            int64_t ex = last != ORC_NONE ? last : c;
            if (ex != ORC_NONE && ex < wn) ex = ORC_NONE;   /* normalise for p + 1 */
            tab[e].cls = c;
            tab[e].count = cnt;
            tab[e].exit = ex;
            e++;
        }
        if (tables_out) tables_out[p] = nent;
        /* Concatenate: look the incoming class up by event index. */
        int64_t hit = -1;
        for (int64_t k = 0; k < nent; k++)
            if (tab[k].cls == cls) { hit = k; break; }
        if (hit < 0) { free(tab); return UINT32_MAX; }
        total += tab[hit].count;
        cls = tab[hit].exit;
        free(tab);
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/*
 * MapConcatenate as the paper prints it (Section 5.2.2), kept as a documented
 * comparison with the exact reformulation above.  Readings (R13):
 *   - segment p holds the events with tau[p] < t <= tau[p+1] (times, not indices);
 *   - machine k (0 <= k < N) of segment p runs Algorithm 1 (pruned lists) on the
 *     events with t > tau[p] - (hi[0] + ... + hi[k-1]);
 *   - it counts the completions with tau[p] < t <= tau[p+1]; a is the end time of
 *     its first completion with tau[p] < t < tau[p] + W (W = sum of hi), else
 *     tau[p];
 *   - past tau[p+1] it only advances the partial occurrences it holds (node 0
 *     admits nothing), over the events with t < tau[p+1] + W; b is the end time
 *     of the first completion there, else tau[p+1];
 *   - Concatenate joins a tuple (a, c, b) of segment p to the tuple of segment
 *     p+1 whose a equals b, starting from machine 0 of segment 0; when several
 *     tuples match it takes the smallest k, when none matches it takes k = 0 and
 *     counts the boundary in diag[0] (diag[1] counts boundaries with several).
 * The paper composes the tuples pairwise in a tree; with a single choice per
 * boundary that composition equals this left-to-right one.
 */

/* Algorithm 1 step with pruned lists; with allow_start == 0 node 0 admits
 * nothing.  Returns 1 on a completion (the lists are then empty). */
static int literal_step(tlist *s, int N, const uint8_t *E, const uint32_t *lo,
                        const uint32_t *hi, uint8_t ty, uint32_t tt, int allow_start,
                        int *oom)
{
    for (int i = N - 1; i >= 0; i--) {
        if (ty != E[i]) continue;
        if (i == 0) {
            if (!allow_start) continue;
            if (N == 1) return 1;
            tlist *L0 = &s[0];
            while (L0->head < L0->len && tt - L0->v[L0->head] > hi[0]) L0->head++;
            if (tl_push(L0, tt)) { *oom = 1; return 0; }
            continue;
        }
        tlist *Q = &s[i - 1];
        while (Q->head < Q->len && tt - Q->v[Q->head] > hi[i - 1]) Q->head++;
        if (!(Q->head < Q->len && tt - Q->v[Q->head] > lo[i - 1])) continue;
        if (i == N - 1) {
            for (int k = 0; k < N; k++) tl_clear(&s[k]);
            return 1;
        }
        tlist *L = &s[i];
        while (L->head < L->len && tt - L->v[L->head] > hi[i]) L->head++;
        if (tl_push(L, tt)) { *oom = 1; return 0; }
    }
    return 0;
}

/* First index j with t[j] > x (n if none). */
static int64_t first_after(const uint32_t *t, int64_t n, int64_t x)
{
    int64_t a = 0, b = n;
    while (a < b) {
        int64_t mid = a + (b - a) / 2;
        if ((int64_t)t[mid] > x) b = mid; else a = mid + 1;
    }
    return a;
}

/*
 * tau: int64[P+1], strictly increasing, tau[0] < t[0], tau[P] >= t[n-1].
 * tuples_out (optional): int64[P*N*3] = (a, count, b) of machine k of segment p
 * at [(p*N + k)*3].  Returns the concatenated count (UINT32_MAX on error).
 */
uint32_t orc_count_mapconcat_literal(const uint8_t *type, const uint32_t *t, int64_t n,
                                     int N, const uint8_t *E, const uint32_t *lo,
                                     const uint32_t *hi, int64_t P, const int64_t *tau,
                                     int64_t *tuples_out, int64_t *diag)
{
    if (P < 1 || N < 1 || N > ORC_LMAX) return UINT32_MAX;
    for (int64_t p = 0; p < P; p++)
        if (tau[p + 1] <= tau[p]) return UINT32_MAX;
    if (n && (tau[0] >= (int64_t)t[0] || tau[P] < (int64_t)t[n - 1])) return UINT32_MAX;
    int64_t W = 0;   /* sum over the N - 1 edges of hi */
    for (int k = 0; k < N - 1; k++) W += hi[k];
    int64_t *tup = (int64_t *)malloc((size_t)(P * N * 3) * sizeof(int64_t));
    if (!tup) return UINT32_MAX;
    int oom = 0;
    for (int64_t p = 0; p < P && !oom; p++) {
        int64_t back = 0;
        for (int k = 0; k < N && !oom; k++) {
            if (k > 0) back += hi[k - 1];
            tlist s[ORC_LMAX];
            memset(s, 0, sizeof(s));
            int64_t cnt = 0, a = tau[p], b = tau[p + 1];
            int have_a = 0;
            for (int64_t j = first_after(t, n, tau[p] - back); j < n; j++) {
                int64_t tj = t[j];
                int phase2 = tj > tau[p + 1];
                if (phase2 && tj >= tau[p + 1] + W) break;
                int done = literal_step(s, N, E, lo, hi, type[j], t[j], !phase2, &oom);
                if (oom) break;
                if (!done) continue;
                if (phase2) { b = tj; break; }
                if (tj > tau[p]) {
                    cnt++;
                    if (!have_a && tj < tau[p] + W) { a = tj; have_a = 1; }
                }
            }
            for (int q = 0; q < ORC_LMAX; q++) tl_free(&s[q]);
            int64_t *o = tup + (p * N + k) * 3;
            o[0] = a; o[1] = cnt; o[2] = b;
        }
    }
    if (oom) { free(tup); return UINT32_MAX; }
    if (tuples_out) memcpy(tuples_out, tup, (size_t)(P * N * 3) * sizeof(int64_t));
    int64_t none = 0, several = 0;
    int64_t total = tup[1];
    int64_t cur_b = tup[2];
    for (int64_t p = 1; p < P; p++) {
        int pick = -1, hits = 0;
        for (int k = 0; k < N; k++)
            if (tup[(p * N + k) * 3] == cur_b) { hits++; if (pick < 0) pick = k; }
        if (hits == 0) { none++; pick = 0; }
        if (hits > 1) several++;
        total += tup[(p * N + pick) * 3 + 1];
        cur_b = tup[(p * N + pick) * 3 + 2];
    }
    free(tup);
    if (diag) { diag[0] = none; diag[1] = several; }
    return (uint32_t)total;
}

/* ------------------------------------------------------------------------ */
/*
 * Window-based frequency, the alternative the paper's Section 2 names (windows of
 * Mannila et al.), with the episode's interval constraints (reading R14): the
 * number of integer window starts s such that the window [s, s + w) holds every
 * event of some occurrence (t[i_1] >= s and t[i_N] < s + w).
 *
 * For each event j that can be the last node, L(j) = the latest first-node time
 * over the occurrences ending at j, by the recurrence over nodes
 *   L_0(j) = t[j];  L_k(j) = max { L_{k-1}(i) : i < j, type[i] = E[k-1],
 *                                  lo[k-1] < t[j] - t[i] <= hi[k-1] }
 * (undefined if the set is empty).  The occurrences ending at j then cover exactly
 * the starts s in (t[j] - w, L(j)], and the count is the size of the union of
 * those ranges over j.
 */
uint64_t orc_count_windows(const uint8_t *type, const uint32_t *t, int64_t n, int N,
                           const uint8_t *E, const uint32_t *lo, const uint32_t *hi,
                           uint32_t w)
{
    if (N < 1 || N > ORC_LMAX || w == 0) return UINT64_MAX;
    int64_t *L = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * (size_t)N * sizeof(int64_t));
    if (!L) return UINT64_MAX;
    for (int64_t q = 0; q < n * N; q++) L[q] = -1;          /* -1: undefined */
    for (int k = 0; k < N; k++) {
        for (int64_t j = 0; j < n; j++) {
            if (type[j] != E[k]) continue;
            if (k == 0) { L[j * N] = t[j]; continue; }
            int64_t best = -1;
            for (int64_t i = j - 1; i >= 0 && t[j] - t[i] <= hi[k - 1]; i--) {
                if (type[i] != E[k - 1] || L[i * N + k - 1] < 0) continue;
                if (t[j] - t[i] <= lo[k - 1]) continue;
                if (L[i * N + k - 1] > best) best = L[i * N + k - 1];
            }
            L[j * N + k] = best;
        }
    }
    uint64_t total = 0;
    int64_t cur_a = 0, cur_b = -1;                          /* merged [cur_a, cur_b] */
    int have = 0;
    for (int64_t j = 0; j < n; j++) {
        int64_t b = L[j * N + N - 1];
        if (type[j] != E[N - 1] || b < 0) continue;
        int64_t a = (int64_t)t[j] - (int64_t)w + 1;
        if (a > b) continue;                                /* occurrence longer than w */
        if (have && a <= cur_b + 1) {
            if (b > cur_b) cur_b = b;
        } else {
            if (have) total += (uint64_t)(cur_b - cur_a + 1);
            cur_a = a; cur_b = b; have = 1;
        }
    }
    if (have) total += (uint64_t)(cur_b - cur_a + 1);
    free(L);
    return total;
}
