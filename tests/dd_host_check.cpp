#include <cstdio>
#include <cmath>
// Host build of the dd phase reduction and sincos that the dd kernels use (dd.cuh is host + device):
// reads "m sh sl" lines (sh, sl as hex floats), prints cos and sin of 2 pi m (sh + sl) as dd hex pairs.
#include "../paper_2304_09139_b300/csrc/dd.cuh"
#define SSH_TABLE_QUAL static
#include "../paper_2304_09139_b300/csrc/gen/tables.h"
int main() {
  double m_, sh, sl;
  while (scanf("%lf %la %la", &m_, &sh, &sl) == 3) {
    ddc z = dd_sincos_turns_tab(dd_turns_times((int)m_, sh, sl), SSH_DD_TAB_A, SSH_DD_TAB_B, SSH_DD_INV_FACT, SSH_DD_2PI);
    printf("%a %a %a %a\n", z.re.hi, z.re.lo, z.im.hi, z.im.lo);
  }
}
