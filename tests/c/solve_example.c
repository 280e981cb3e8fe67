/* Plain-C client of libtw: exact treewidth of a 5-cycle with a chord and of
 * the 3x3 grid through tw_solve, and one decide call, using only include/tw.h.
 * Prints one line per graph; exit status 0 when every answer is the known
 * value (cycle with a chord: 2; 3x3 grid: 3; decide(grid, 2) = no). */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "tw.h"

static void add_edge(uint64_t* rows, int u, int v) {
  rows[u] |= 1ull << v;
  rows[v] |= 1ull << u;
}

int main(void) {
  tw_ctx* ctx = NULL;
  tw_config cfg;
  memset(&cfg, 0, sizeof(cfg));
  int rc = tw_create(&ctx, &cfg);
  if (rc != TW_OK) {
    printf("tw_create: %s\n", tw_strerror(rc));
    return 1;
  }
  int failures = 0;

  uint64_t cyc[5] = {0};
  for (int v = 0; v < 5; ++v) add_edge(cyc, v, (v + 1) % 5);
  add_edge(cyc, 0, 2);
  int tw = -1;
  int32_t order[9];
  rc = tw_solve(ctx, cyc, 5, &tw, order, NULL, NULL, NULL);
  printf("cycle5+chord: status %d tw %d\n", rc, tw);
  failures += (rc != TW_OK || tw != 2);

  uint64_t grid[9] = {0};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      if (c < 2) add_edge(grid, 3 * r + c, 3 * r + c + 1);
      if (r < 2) add_edge(grid, 3 * r + c, 3 * r + c + 3);
    }
  tw_stats st;
  rc = tw_solve(ctx, grid, 9, &tw, order, NULL, NULL, &st);
  printf("grid3x3: status %d tw %d states %llu\n", rc, tw, (unsigned long long)st.states_expanded);
  failures += (rc != TW_OK || tw != 3);

  int yes = -1;
  rc = tw_decide(ctx, grid, 9, 2, &yes, NULL, NULL);
  printf("grid3x3 decide(2): status %d yes %d\n", rc, yes);
  failures += (rc != TW_OK || yes != 0);

  tw_destroy(ctx);
  return failures ? 1 : 0;
}
