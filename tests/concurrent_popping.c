/*
 * Several threads sample ONE Wilson run together (test infrastructure: the
 * protocol of test_oracle_concurrent_popping.py under real races, with the
 * node-word layout planned for a GPU kernel).
 *
 * word[u] (64 bits, updated with compare-and-swap):
 *   bit 63 InTree | bits 57..62 owner (walker + 1, 0 = free) | bit 56 pending |
 *   bits 32..55 draws k | bits 0..31 arrow (a path's next node, or the arrow an
 *   aborted walker left pending; 0xFFFFFFFF none)
 *
 * A walker only ever writes words of nodes it owns, except to claim a free
 * node (CAS from the word it read).  Draw j of node u is draws[u * kmax + j],
 * computed by the caller (the oracle's Philox keying); a draw index >= kmax
 * is reported as an error.  Waits go from lower- to higher-numbered walkers
 * only, so they cannot form a cycle.
 */
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>

#define IN_TREE (1ull << 63)
#define OWNER_SHIFT 57
#define OWNER_MASK (63ull << OWNER_SHIFT)
#define PENDING (1ull << 56)
#define K_SHIFT 32
#define K_MASK (0xFFFFFFull << K_SHIFT)
#define NONE 0xFFFFFFFFu

typedef struct {
    int32_t n, v, kmax, walkers;
    const int32_t *draws;
    _Atomic uint64_t *word;
    atomic_int remaining;
    atomic_int error;
    atomic_long steps;
    long step_limit;
} shared_t;

typedef struct {
    shared_t *sh;
    int id;               /* walker number, owner field = id + 1 */
    uint64_t rng;         /* xorshift state for random yields */
    int32_t *path;
} walker_t;

static uint32_t arrow_of(uint64_t w) { return (uint32_t)w; }
static uint32_t owner_of(uint64_t w) { return (uint32_t)((w & OWNER_MASK) >> OWNER_SHIFT); }
static uint32_t k_of(uint64_t w) { return (uint32_t)((w & K_MASK) >> K_SHIFT); }
static uint64_t make(int intree, uint32_t owner, int pending, uint32_t k, uint32_t arrow)
{
    return (intree ? IN_TREE : 0) | ((uint64_t)owner << OWNER_SHIFT) | (pending ? PENDING : 0) |
           ((uint64_t)k << K_SHIFT) | arrow;
}

static void maybe_yield(walker_t *me)
{
    uint64_t x = me->rng;
    x ^= x << 13; x ^= x >> 7; x ^= x << 17;
    me->rng = x;
    if ((x & 7) == 0) sched_yield();
}

static void *walk(void *arg)
{
    walker_t *me = (walker_t *)arg;
    shared_t *sh = me->sh;
    const uint32_t self = (uint32_t)me->id + 1u;
    int32_t len = 0;
    int32_t scan = 0;
    while (atomic_load(&sh->remaining) > 0 && !atomic_load(&sh->error)) {
        if (atomic_fetch_add(&sh->steps, 1) > sh->step_limit) { atomic_store(&sh->error, 2); break; }
        maybe_yield(me);
        if (len == 0) {
            /* Claim a start: the next free, non-tree node from the scan position. */
            for (int32_t t = 0; t < sh->n && len == 0; ++t) {
                const int32_t u = (scan + t) % sh->n;
                uint64_t w = atomic_load(&sh->word[u]);
                if ((w & IN_TREE) || owner_of(w)) continue;
                if (atomic_compare_exchange_strong(&sh->word[u], &w, w | ((uint64_t)self << OWNER_SHIFT))) {
                    me->path[len++] = u;
                    scan = u;
                }
            }
            continue;
        }
        const int32_t u = me->path[len - 1];
        uint64_t wu = atomic_load(&sh->word[u]);          /* owned: no one else writes it */
        if (arrow_of(wu) == NONE || (wu & PENDING)) {
            if (wu & PENDING) {
                wu = make(0, self, 0, k_of(wu), arrow_of(wu));
            } else {
                const uint32_t k = k_of(wu);
                if ((int32_t)k >= sh->kmax) { atomic_store(&sh->error, 1); break; }
                wu = make(0, self, 0, k + 1u, (uint32_t)sh->draws[(int64_t)u * sh->kmax + k]);
            }
            atomic_store(&sh->word[u], wu);
        }
        const int32_t w = (int32_t)arrow_of(wu);
        uint64_t ww = atomic_load(&sh->word[w]);
        if (ww & IN_TREE) {
            /* The loop-erased path joins the tree. */
            for (int32_t j = 0; j < len; ++j) {
                const int32_t x = me->path[j];
                const uint64_t wx = atomic_load(&sh->word[x]);
                atomic_store(&sh->word[x], make(1, 0, 0, k_of(wx), arrow_of(wx)));
            }
            atomic_fetch_sub(&sh->remaining, len);
            len = 0;
        } else if (owner_of(ww) == self) {
            /* A cycle of stack tops closed at w: pop it (its arrows are consumed). */
            while (me->path[len - 1] != w) {
                const int32_t x = me->path[--len];
                const uint64_t wx = atomic_load(&sh->word[x]);
                atomic_store(&sh->word[x], make(0, 0, 0, k_of(wx), NONE));
            }
            atomic_store(&sh->word[w], make(0, self, 0, k_of(ww), NONE));
        } else if (owner_of(ww)) {
            if (self > owner_of(ww)) {
                /* Abort: leave every arrow of the path pending on its node. */
                for (int32_t j = 0; j < len; ++j) {
                    const int32_t x = me->path[j];
                    const uint64_t wx = atomic_load(&sh->word[x]);
                    atomic_store(&sh->word[x], make(0, 0, 1, k_of(wx), arrow_of(wx)));
                }
                len = 0;
            }
            /* else wait: the same arrow is tried again */
        } else {
            if (atomic_compare_exchange_strong(&sh->word[w], &ww, ww | ((uint64_t)self << OWNER_SHIFT)))
                me->path[len++] = w;
        }
    }
    return NULL;
}

/*
 * Runs one Wilson sample with `walkers` threads.  draws: n * kmax node ids.
 * Outputs k[n] (draws per node = visits) and arrow[n] (tree parent; v: -1).
 * Returns 0, 1 (a draw index reached kmax), 2 (step limit) or 3 (thread error).
 */
int concurrent_popping(int32_t n, int32_t v, int32_t kmax, const int32_t *draws, int32_t walkers,
                       uint64_t yield_seed, long step_limit, int32_t *k_out, int32_t *arrow_out)
{
    shared_t sh;
    sh.n = n; sh.v = v; sh.kmax = kmax; sh.walkers = walkers; sh.draws = draws;
    sh.step_limit = step_limit;
    sh.word = (_Atomic uint64_t *)malloc(sizeof(_Atomic uint64_t) * (size_t)n);
    for (int32_t u = 0; u < n; ++u) atomic_init(&sh.word[u], make(u == v, 0, 0, 0, NONE));
    atomic_init(&sh.remaining, n - 1);
    atomic_init(&sh.error, 0);
    atomic_init(&sh.steps, 0);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)walkers);
    walker_t *wk = (walker_t *)malloc(sizeof(walker_t) * (size_t)walkers);
    int rc = 0;
    int started = 0;
    for (int i = 0; i < walkers; ++i) {
        wk[i].sh = &sh;
        wk[i].id = i;
        wk[i].rng = yield_seed * 0x9E3779B97F4A7C15ull + (uint64_t)i + 1u;
        wk[i].path = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        if (pthread_create(&th[i], NULL, walk, &wk[i]) != 0) { rc = 3; atomic_store(&sh.error, 3); break; }
        ++started;
    }
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    if (!rc) rc = atomic_load(&sh.error);
    for (int32_t u = 0; u < n; ++u) {
        const uint64_t w = atomic_load(&sh.word[u]);
        k_out[u] = (int32_t)k_of(w);
        arrow_out[u] = u == v ? -1 : (int32_t)arrow_of(w);
    }
    for (int i = 0; i < walkers; ++i) free(wk[i].path);
    free(wk); free(th); free((void *)sh.word);
    return rc;
}
