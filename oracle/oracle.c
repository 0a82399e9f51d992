/*
 * CPU oracle for strong-bisimulation partition refinement.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain, single-threaded
 * reference the CUDA path is checked against. Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the library never
 * does. It shares no code, header or table with the CUDA sources.
 *
 * Functions (all return 0 on success, a negative value on bad input):
 *
 *  oracle_ks       Kanellakis-Smolka refinement with a FIFO of unstable
 *                  blocks (Section 3.1, Algorithm 1), generalised to action
 *                  labels by splitting on pre_a(B) for every action a.
 *                  Returns canonical block ids (first occurrence order).
 *
 *  oracle_plan     The preprocessing arrays of Section 4.1.1: transitions
 *                  sorted by (source, a), action_switch (Algorithm 4),
 *                  order (segmented prefix sum), nr_marks, off, mark_length.
 *
 *  oracle_pram     Lock-step simulation of the PRAM program under the
 *                  priority write rule (lowest processor index wins):
 *                  initial leaders (Algorithm 2, lines 1-6), the action-set
 *                  preprocessing (Algorithm 5, one round per label that
 *                  occurs, in increasing label order) and the main loop of
 *                  Algorithm 3 (or Algorithm 2 when alg2 != 0, |Act| = 1).
 *                  Returns the raw block labels (leader indices) and the
 *                  number of while-loop iterations, counting the final
 *                  iteration in which no splitter is found.
 *
 *  oracle_pram_step  One iteration of the main loop with a given splitter C
 *                  (used to replay the worked example of Figure 1).
 *
 *  oracle_pair     (C, a)-pair splitters: Algorithm 2 applied with one action
 *                  label at a time. The priority rule picks the smallest
 *                  unstable label C; then one iteration per label a that
 *                  occurs, in increasing order, marks the states with an
 *                  a-transition into C (one flag per state), splits every
 *                  block into the states whose flag equals the leader's and
 *                  the rest, and elects the smallest state of the rest as its
 *                  leader; both labels of a split block become unstable (as
 *                  in Algorithm 2, the splitter is not set unstable again).
 *                  No action-set preprocessing is needed: the first
 *                  selection of every block splits it by each label. With a
 *                  single label this is Algorithm 2 exactly. Returns the raw
 *                  block labels and the number of iterations, one per
 *                  (C, a) pair plus the final one that finds no splitter.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_EROUNDS (-4)

static int check_input(int32_t n, int64_t m, int32_t A, const int32_t* src, const int32_t* act,
                       const int32_t* dst, const int32_t* init) {
    if (n < 0 || m < 0 || A < 1) return OR_EINVAL;
    for (int64_t i = 0; i < m; i++) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return OR_EINVAL;
        if (act && (act[i] < 0 || act[i] >= A)) return OR_EINVAL;
    }
    if (init)
        for (int32_t s = 0; s < n; s++)
            if (init[s] < 0 || init[s] >= n) return OR_EINVAL;
    return 0;
}

/* Canonical numbering: block ids in order of their first state. */
static void canonical(int32_t n, const int32_t* label, int32_t* out, int32_t* scratch) {
    for (int32_t i = 0; i < n; i++) scratch[i] = -1;
    int32_t next = 0;
    for (int32_t s = 0; s < n; s++) {
        int32_t b = label[s];
        if (scratch[b] < 0) scratch[b] = next++;
        out[s] = scratch[b];
    }
}

/* ------------------------------------------------------------------------- */
/* Kanellakis-Smolka with a refinable partition.                               */
/* ------------------------------------------------------------------------- */

typedef struct { int32_t a, s; } pair_t;

static int cmp_pair(const void* x, const void* y) {
    const pair_t* p = (const pair_t*)x;
    const pair_t* q = (const pair_t*)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->s != q->s) return p->s < q->s ? -1 : 1;
    return 0;
}

int oracle_ks(int32_t n, int64_t m, int32_t A, const int32_t* src, const int32_t* act,
              const int32_t* dst, const int32_t* init, int32_t* out, int64_t* stats) {
    int rc = check_input(n, m, A, src, act, dst, init);
    if (rc) return rc;
    if (n == 0) return 0;
    int64_t* in_ptr = calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* in_src = malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    int32_t* in_act = malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    int32_t* elems = malloc(sizeof(int32_t) * (size_t)n);
    int32_t* loc = malloc(sizeof(int32_t) * (size_t)n);
    int32_t* blk = malloc(sizeof(int32_t) * (size_t)n);
    int32_t* bbeg = malloc(sizeof(int32_t) * (size_t)n);
    int32_t* bend = malloc(sizeof(int32_t) * (size_t)n);
    int32_t* bmark = calloc((size_t)n, sizeof(int32_t));
    int32_t* queue = malloc(sizeof(int32_t) * (size_t)n);
    char* inq = calloc((size_t)n, 1);
    int32_t* touched = malloc(sizeof(int32_t) * (size_t)n);
    int32_t* scratch = malloc(sizeof(int32_t) * (size_t)n);
    size_t pcap = 1024;
    pair_t* pairs = malloc(sizeof(pair_t) * pcap);
    if (!in_ptr || !in_src || !in_act || !elems || !loc || !blk || !bbeg || !bend || !bmark ||
        !queue || !inq || !touched || !scratch || !pairs) {
        rc = OR_ENOMEM;
        goto done;
    }
    /* in-transition index by target (counting sort) */
    for (int64_t i = 0; i < m; i++) in_ptr[dst[i] + 1]++;
    for (int32_t t = 0; t < n; t++) in_ptr[t + 1] += in_ptr[t];
    {
        int64_t* fill = malloc(sizeof(int64_t) * (size_t)n);
        if (!fill) { rc = OR_ENOMEM; goto done; }
        memcpy(fill, in_ptr, sizeof(int64_t) * (size_t)n);
        for (int64_t i = 0; i < m; i++) {
            int64_t p = fill[dst[i]]++;
            in_src[p] = src[i];
            in_act[p] = act ? act[i] : 0;
        }
        free(fill);
    }
    /* initial partition: one block per distinct initial label, states in
       increasing order inside each block */
    int32_t nb = 0;
    {
        int32_t* cnt = calloc((size_t)n, sizeof(int32_t));
        int32_t* id = malloc(sizeof(int32_t) * (size_t)n);
        if (!cnt || !id) { free(cnt); free(id); rc = OR_ENOMEM; goto done; }
        for (int32_t s = 0; s < n; s++) cnt[init ? init[s] : 0]++;
        int32_t pos = 0;
        for (int32_t v = 0; v < n; v++) {
            id[v] = -1;
            if (cnt[v]) {
                id[v] = nb;
                bbeg[nb] = pos;
                bend[nb] = pos;
                pos += cnt[v];
                nb++;
            }
        }
        for (int32_t s = 0; s < n; s++) {
            int32_t b = id[init ? init[s] : 0];
            blk[s] = b;
            elems[bend[b]] = s;
            loc[s] = bend[b];
            bend[b]++;
        }
        free(cnt);
        free(id);
    }
    int64_t qh = 0, qt = 0; /* FIFO over a ring of n slots; a block is queued at most once */
    for (int32_t b = 0; b < nb; b++) { queue[qt++ % n] = b; inq[b] = 1; }
    int64_t pops = 0, splits = 0;
    while (qh < qt) {
        int32_t B = queue[qh++ % n];
        inq[B] = 0;
        pops++;
        /* snapshot: all (a, s) with s -a-> t for a member t of B */
        size_t np = 0;
        for (int32_t k = bbeg[B]; k < bend[B]; k++) {
            int32_t t = elems[k];
            for (int64_t j = in_ptr[t]; j < in_ptr[t + 1]; j++) {
                if (np == pcap) {
                    pcap *= 2;
                    pair_t* np2 = realloc(pairs, sizeof(pair_t) * pcap);
                    if (!np2) { rc = OR_ENOMEM; goto done; }
                    pairs = np2;
                }
                pairs[np].a = in_act[j];
                pairs[np].s = in_src[j];
                np++;
            }
        }
        qsort(pairs, np, sizeof(pair_t), cmp_pair);
        size_t g = 0;
        while (g < np) {
            /* S'_a = pre_a(B) for the action of this group */
            size_t h = g;
            int32_t nt = 0;
            while (h < np && pairs[h].a == pairs[g].a) {
                if (h == g || pairs[h].s != pairs[h - 1].s) {
                    int32_t s = pairs[h].s;
                    int32_t b = blk[s];
                    /* move s into the marked prefix of its block */
                    int32_t p = bbeg[b] + bmark[b];
                    int32_t other = elems[p];
                    int32_t ls = loc[s];
                    elems[p] = s; loc[s] = p;
                    elems[ls] = other; loc[other] = ls;
                    if (bmark[b] == 0) touched[nt++] = b;
                    bmark[b]++;
                }
                h++;
            }
            /* split every B' with 0 < |B' n S'| < |B'| */
            for (int32_t i = 0; i < nt; i++) {
                int32_t b = touched[i];
                int32_t k = bmark[b];
                bmark[b] = 0;
                if (k == bend[b] - bbeg[b]) continue;
                int32_t nw = nb++;
                bbeg[nw] = bbeg[b];
                bend[nw] = bbeg[b] + k;
                bbeg[b] = bbeg[b] + k;
                for (int32_t q = bbeg[nw]; q < bend[nw]; q++) blk[elems[q]] = nw;
                splits++;
                if (!inq[b]) { queue[qt++ % n] = b; inq[b] = 1; }
                queue[qt++ % n] = nw;
                inq[nw] = 1;
            }
            g = h;
        }
    }
    canonical(n, blk, out, scratch);
    if (stats) { stats[0] = pops; stats[1] = splits; stats[2] = nb; }
done:
    free(in_ptr); free(in_src); free(in_act); free(elems); free(loc); free(blk); free(bbeg);
    free(bend); free(bmark); free(queue); free(inq); free(touched); free(scratch); free(pairs);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Preprocessing of Section 4.1.1                                             */
/* ------------------------------------------------------------------------- */

typedef struct { int32_t s, a; int64_t i; } tr_t;

static int cmp_tr(const void* x, const void* y) {
    const tr_t* p = (const tr_t*)x;
    const tr_t* q = (const tr_t*)y;
    if (p->s != q->s) return p->s < q->s ? -1 : 1;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->i != q->i) return p->i < q->i ? -1 : 1;
    return 0;
}

/* perm[k]      index of the k-th transition in (source, a) order
 * action_switch[k], order[k]  for the k-th sorted transition
 * nr_marks[s], off[s]  per state; off is the exclusive prefix sum of nr_marks
 * *mark_length  sum of nr_marks */
int oracle_plan(int32_t n, int64_t m, int32_t A, const int32_t* src, const int32_t* act,
                const int32_t* dst, int64_t* perm, int32_t* action_switch, int32_t* order,
                int32_t* nr_marks, int64_t* off, int64_t* mark_length) {
    int rc = check_input(n, m, A, src, act, dst, NULL);
    if (rc) return rc;
    tr_t* t = malloc(sizeof(tr_t) * (size_t)(m ? m : 1));
    if (!t) return OR_ENOMEM;
    for (int64_t i = 0; i < m; i++) { t[i].s = src[i]; t[i].a = act ? act[i] : 0; t[i].i = i; }
    qsort(t, (size_t)m, sizeof(tr_t), cmp_tr);
    /* Algorithm 4: a switch is a change of label within the same source */
    for (int64_t k = 0; k < m; k++) {
        perm[k] = t[k].i;
        if (k == 0 || t[k].s != t[k - 1].s || t[k].a == t[k - 1].a)
            action_switch[k] = 0;
        else
            action_switch[k] = 1;
    }
    /* order: prefix sum of action_switch restarted at every new source */
    for (int64_t k = 0; k < m; k++) {
        if (k == 0 || t[k].s != t[k - 1].s)
            order[k] = action_switch[k];
        else
            order[k] = order[k - 1] + action_switch[k];
    }
    /* nr_marks: number of distinct labels of the source = last order + 1 */
    for (int32_t s = 0; s < n; s++) nr_marks[s] = 0;
    for (int64_t k = 0; k < m; k++)
        if (k == m - 1 || t[k + 1].s != t[k].s) nr_marks[t[k].s] = order[k] + 1;
    int64_t acc = 0;
    for (int32_t s = 0; s < n; s++) { off[s] = acc; acc += nr_marks[s]; }
    *mark_length = acc;
    free(t);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Lock-step PRAM simulation, priority rule                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t n; int64_t m; int32_t A;
    int64_t* perm; int32_t* sw; int32_t* order; int32_t* nr; int64_t* off; int64_t L;
    int32_t *ssrc, *sact, *sdst; /* transitions in sorted order */
    char* mark; char* split; char* unstable; int32_t* new_leader; int32_t* block;
} pram_t;

static void pram_free(pram_t* p) {
    free(p->perm); free(p->sw); free(p->order); free(p->nr); free(p->off);
    free(p->ssrc); free(p->sact); free(p->sdst);
    free(p->mark); free(p->split); free(p->unstable); free(p->new_leader); free(p->block);
}

static int pram_init(pram_t* p, int32_t n, int64_t m, int32_t A, const int32_t* src,
                     const int32_t* act, const int32_t* dst) {
    memset(p, 0, sizeof(*p));
    p->n = n; p->m = m; p->A = A;
    size_t mm = (size_t)(m ? m : 1), nn = (size_t)(n ? n : 1);
    p->perm = malloc(sizeof(int64_t) * mm);
    p->sw = malloc(sizeof(int32_t) * mm);
    p->order = malloc(sizeof(int32_t) * mm);
    p->nr = malloc(sizeof(int32_t) * nn);
    p->off = malloc(sizeof(int64_t) * nn);
    p->ssrc = malloc(sizeof(int32_t) * mm);
    p->sact = malloc(sizeof(int32_t) * mm);
    p->sdst = malloc(sizeof(int32_t) * mm);
    p->split = malloc(nn);
    p->unstable = malloc(nn);
    p->new_leader = malloc(sizeof(int32_t) * nn);
    p->block = malloc(sizeof(int32_t) * nn);
    if (!p->perm || !p->sw || !p->order || !p->nr || !p->off || !p->ssrc || !p->sact || !p->sdst ||
        !p->split || !p->unstable || !p->new_leader || !p->block)
        return OR_ENOMEM;
    int rc = oracle_plan(n, m, A, src, act, dst, p->perm, p->sw, p->order, p->nr, p->off, &p->L);
    if (rc) return rc;
    p->mark = malloc((size_t)(p->L > n ? p->L : n) + 1); /* slot marks or state marks */
    if (!p->mark) return OR_ENOMEM;
    for (int64_t k = 0; k < m; k++) {
        int64_t i = p->perm[k];
        p->ssrc[k] = src[i];
        p->sact[k] = act ? act[i] : 0;
        p->sdst[k] = dst[i];
    }
    return 0;
}

/* Lock-step leader election under the priority rule: every processor i in
   `who` writes i to new_leader[block_i]; the lowest index wins. Then every
   such processor reads new_leader[block_i] as its new block. */
static void elect_and_relabel(pram_t* p, const char* who, char* unstable, int32_t C, int alg2) {
    int32_t n = p->n;
    for (int32_t i = n - 1; i >= 0; i--)       /* lowest index wins = last write */
        if (who[i]) p->new_leader[p->block[i]] = i;
    if (unstable) {
        int any = 0;
        for (int32_t i = 0; i < n; i++)
            if (who[i]) { unstable[p->block[i]] = 1; any = 1; }
        for (int32_t i = 0; i < n; i++)
            if (who[i]) p->block[i] = p->new_leader[p->block[i]];
        for (int32_t i = 0; i < n; i++)
            if (who[i]) unstable[p->block[i]] = 1;
        if (any && !alg2) unstable[C] = 1;
    } else {
        for (int32_t i = 0; i < n; i++)
            if (who[i]) p->block[i] = p->new_leader[p->block[i]];
    }
}

/* One main-loop iteration with splitter C (C >= 0). mark_out, if given,
   receives the mark list (mark_length entries) after the marking step. */
static void pram_iteration(pram_t* p, int32_t C, int alg2, char* mark_out) {
    int32_t n = p->n;
    memset(p->split, 0, (size_t)n);
    if (alg2) {
        /* Algorithm 2: one mark per state; split when it differs from the
           leader's mark */
        memset(p->mark, 0, (size_t)n);
        for (int64_t k = 0; k < p->m; k++)
            if (p->block[p->sdst[k]] == C) p->mark[p->ssrc[k]] = 1;
        if (mark_out) memcpy(mark_out, p->mark, (size_t)n);
        for (int32_t i = 0; i < n; i++) p->split[i] = p->mark[i] != p->mark[p->block[i]];
    } else {
        /* Algorithm 3: one mark per (state, label) pair at off(s) + order */
        memset(p->mark, 0, (size_t)p->L + 1);
        for (int64_t k = 0; k < p->m; k++)
            if (p->block[p->sdst[k]] == C) p->mark[p->off[p->ssrc[k]] + p->order[k]] = 1;
        if (mark_out) memcpy(mark_out, p->mark, (size_t)p->L);
        for (int64_t k = 0; k < p->m; k++) {
            int32_t s = p->ssrc[k];
            if (p->mark[p->off[s] + p->order[k]] != p->mark[p->off[p->block[s]] + p->order[k]])
                p->split[s] = 1;
        }
    }
    p->unstable[C] = 0;
    elect_and_relabel(p, p->split, p->unstable, C, alg2);
}

static void pram_initial(pram_t* p, const int32_t* init) {
    int32_t n = p->n;
    char* all = malloc((size_t)(n ? n : 1));
    for (int32_t i = 0; i < n; i++) { all[i] = 1; p->block[i] = init ? init[i] : 0; }
    /* new_leader[I_i] := i (priority), block_i := new_leader[I_i] */
    elect_and_relabel(p, all, NULL, 0, 1);
    free(all);
}

/* Action-set preprocessing (Algorithm 5): one round per label that occurs,
   in increasing label order. Returns the number of rounds. */
static int64_t pram_preprocess(pram_t* p) {
    int32_t n = p->n;
    char* used = calloc((size_t)p->A, 1);
    for (int64_t k = 0; k < p->m; k++) used[p->sact[k]] = 1;
    int64_t rounds = 0;
    for (int32_t a = 0; a < p->A; a++) {
        if (!used[a]) continue;
        rounds++;
        memset(p->mark, 0, (size_t)n);
        for (int64_t k = 0; k < p->m; k++)
            if (p->sact[k] == a) p->mark[p->ssrc[k]] = 1;
        for (int32_t i = 0; i < n; i++) p->split[i] = p->mark[i] != p->mark[p->block[i]];
        elect_and_relabel(p, p->split, NULL, 0, 1);
    }
    free(used);
    return rounds;
}

int oracle_pram(int32_t n, int64_t m, int32_t A, const int32_t* src, const int32_t* act,
                const int32_t* dst, const int32_t* init, int32_t alg2, int32_t skip_preprocess,
                int64_t round_cap, int32_t* out_labels, int64_t* out_rounds,
                int64_t* out_pre_rounds) {
    int rc = check_input(n, m, A, src, act, dst, init);
    if (rc) return rc;
    if (alg2 && A != 1) return OR_EINVAL;
    pram_t p;
    rc = pram_init(&p, n, m, A, src, act, dst);
    if (rc) { pram_free(&p); return rc; }
    pram_initial(&p, init);
    int64_t pre = skip_preprocess ? 0 : pram_preprocess(&p);
    /* Algorithm 3, lines 1-3 */
    for (int32_t i = 0; i < n; i++) p.unstable[i] = 0;
    for (int32_t i = 0; i < n; i++) p.unstable[p.block[i]] = 1;
    int64_t rounds = 0;
    for (;;) {
        rounds++;
        if (round_cap > 0 && rounds > round_cap) { rc = OR_EROUNDS; break; }
        int32_t C = -1;
        for (int32_t i = 0; i < n; i++)
            if (p.unstable[i]) { C = i; break; } /* lowest writer wins */
        if (C < 0) break;
        pram_iteration(&p, C, alg2, NULL);
    }
    memcpy(out_labels, p.block, sizeof(int32_t) * (size_t)n);
    *out_rounds = rounds;
    *out_pre_rounds = pre;
    pram_free(&p);
    return rc;
}

/* One iteration from a given state: block_inout / unstable_inout hold the
   partition (leader labels) and the unstable flags before the iteration and
   receive them afterwards; marks_out receives the marks after the marking
   step: one per state (n entries) when alg2 != 0, else the mark list of
   mark_length entries. */
int oracle_pram_step(int32_t n, int64_t m, int32_t A, const int32_t* src, const int32_t* act,
                     const int32_t* dst, int32_t* block_inout, int8_t* unstable_inout,
                     int32_t C, int32_t alg2, int8_t* marks_out, int64_t* mark_length) {
    int rc = check_input(n, m, A, src, act, dst, block_inout);
    if (rc) return rc;
    if (C < 0 || C >= n) return OR_EINVAL;
    pram_t p;
    rc = pram_init(&p, n, m, A, src, act, dst);
    if (rc) { pram_free(&p); return rc; }
    memcpy(p.block, block_inout, sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; i++) p.unstable[i] = unstable_inout[i] != 0;
    pram_iteration(&p, C, alg2, (char*)marks_out);
    memcpy(block_inout, p.block, sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; i++) unstable_inout[i] = p.unstable[i];
    *mark_length = p.L;
    pram_free(&p);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* (C, a)-pair splitters                                                       */
/* ------------------------------------------------------------------------- */

int oracle_pair(int32_t n, int64_t m, int32_t A, const int32_t* src, const int32_t* act,
                const int32_t* dst, const int32_t* init, int64_t round_cap, int32_t* out_labels,
                int64_t* out_rounds) {
    int rc = check_input(n, m, A, src, act, dst, init);
    if (rc) return rc;
    size_t nn = (size_t)(n ? n : 1);
    int32_t* block = malloc(sizeof(int32_t) * nn);
    int32_t* leader = malloc(sizeof(int32_t) * nn);
    char* mark = malloc(nn);
    char* split = malloc(nn);
    char* unstable = malloc(nn);
    char* occurs = calloc((size_t)A, 1);
    if (!block || !leader || !mark || !split || !unstable || !occurs) {
        free(block); free(leader); free(mark); free(split); free(unstable); free(occurs);
        return OR_ENOMEM;
    }
    for (int64_t k = 0; k < m; k++) occurs[act ? act[k] : 0] = 1;
    /* initial leaders: the smallest state of every initial block */
    for (int32_t i = 0; i < n; i++) leader[i] = -1;
    for (int32_t i = 0; i < n; i++) {
        int32_t b = init ? init[i] : 0;
        if (leader[b] < 0) leader[b] = i;
    }
    for (int32_t i = 0; i < n; i++) block[i] = leader[init ? init[i] : 0];
    for (int32_t i = 0; i < n; i++) unstable[i] = block[i] == i;
    int32_t nlab = 0;
    for (int32_t a = 0; a < A; a++) nlab += occurs[a];
    int64_t rounds = 0;
    for (;;) {
        rounds++;
        if (round_cap > 0 && rounds > round_cap) { rc = OR_EROUNDS; break; }
        int32_t C = -1;
        for (int32_t i = 0; i < n; i++)
            if (unstable[i]) { C = i; break; }
        if (C < 0) break;
        unstable[C] = 0;
        int32_t done = 0;
        for (int32_t a = 0; a < A; a++) {
            if (!occurs[a]) continue;
            if (done++ > 0) {
                rounds++;
                if (round_cap > 0 && rounds > round_cap) { rc = OR_EROUNDS; break; }
            }
            /* mark: s -a-> t with t in C */
            memset(mark, 0, nn);
            for (int64_t k = 0; k < m; k++)
                if ((act ? act[k] : 0) == a && block[dst[k]] == C) mark[src[k]] = 1;
            /* split: the flag differs from the leader's */
            for (int32_t i = 0; i < n; i++) split[i] = mark[i] != mark[block[i]];
            /* priority election of the new leader, then relabelling */
            for (int32_t i = n - 1; i >= 0; i--)
                if (split[i]) leader[block[i]] = i;
            for (int32_t i = 0; i < n; i++)
                if (split[i]) unstable[block[i]] = 1;
            for (int32_t i = 0; i < n; i++)
                if (split[i]) block[i] = leader[block[i]];
            for (int32_t i = 0; i < n; i++)
                if (split[i]) unstable[block[i]] = 1;
        }
        if (rc) break;
    }
    memcpy(out_labels, block, sizeof(int32_t) * (size_t)n);
    *out_rounds = rounds;
    free(block); free(leader); free(mark); free(split); free(unstable); free(occurs);
    return rc;
}
