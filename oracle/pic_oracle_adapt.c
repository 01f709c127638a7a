/*
 * ORACLE -- test infrastructure only (see pic_oracle.c).
 *
 * 2:1 balance of a mesh adaptation (§3.1 refinement / coarsening of the cell-based AMR grid,
 * §4.3 AMR as particle management).  Each leaf has a target level T = level + 1 (refine),
 * level - 1 (member of a sibling quartet that coarsens) or level.  Two leaves that touch
 * across a face or a corner must end with targets that differ by at most one.  Refinement
 * wins: a leaf whose target is more than one below a touching leaf's target is refined, or,
 * if it was coarsening, its quartet stays.  Every such change is forced, so repeating until
 * nothing changes gives the least balanced set of targets above the requested one.
 */
#include <stdint.h>

typedef struct {
    int32_t nx0, ny0, lmax, bc_x, bc_y;
    int32_t pad_;
    double h0;
    int64_t nleaf;
    const int64_t *key;
    const int32_t *ix, *iy, *s;
} or_mesh;

int64_t or_leaf_at(const or_mesh *m, int32_t I, int32_t J);

static int32_t target(int64_t i, const int32_t *level, const int32_t *refine, const int64_t *group,
                      const int32_t *gactive)
{
    int32_t t = level[i] + (refine[i] ? 1 : 0);
    if (group[i] >= 0 && gactive[group[i]]) t -= 1;
    return t;
}

/* refine[i], gactive[g] are updated in place; group[i] = index of the first leaf of i's
 * coarsening quartet or -1.  Returns the number of sweeps. */
int32_t or_adapt_balance(const or_mesh *m, const int32_t *level, int32_t *refine, const int64_t *group,
                         int32_t *gactive)
{
    int32_t sweeps = 0;
    int changed = 1;
    while (changed) {
        changed = 0;
        ++sweeps;
        for (int64_t a = 0; a < m->nleaf; ++a) {
            int32_t x = m->ix[a], y = m->iy[a], s = m->s[a];
            /* lattice cells just outside the leaf: both ends of each face and the 4 corners */
            int32_t P[12][2] = {{x - 1, y}, {x - 1, y + s - 1}, {x + s, y}, {x + s, y + s - 1},
                                {x, y - 1}, {x + s - 1, y - 1}, {x, y + s}, {x + s - 1, y + s},
                                {x - 1, y - 1}, {x + s, y - 1}, {x - 1, y + s}, {x + s, y + s}};
            int32_t ta = target(a, level, refine, group, gactive);
            for (int k = 0; k < 12; ++k) {
                int64_t b = or_leaf_at(m, P[k][0], P[k][1]);
                if (b < 0 || b == a) continue;
                if (group[a] >= 0 && group[a] == group[b]) continue;
                int32_t tb = target(b, level, refine, group, gactive);
                if (ta < tb - 1) {
                    if (group[a] >= 0 && gactive[group[a]]) gactive[group[a]] = 0;
                    else if (!refine[a] && level[a] < m->lmax) refine[a] = 1;
                    else continue;
                    changed = 1;
                    ta = target(a, level, refine, group, gactive);
                }
            }
        }
    }
    return sweeps;
}
