// Runs the library's FP64 geometry and BF16 rounding helpers (host-device
// functions of csrc/common.cuh) on the host, for tests/test_host_helpers.py.
// Reads commands from stdin, one per line, doubles in C99 hex notation:
//   bf16 x                      -> the 16-bit code of srt_f64_to_bf16(x)
//   arc cx cy r x0 x1 y0 y1     -> srt_arc_in_rect, then srt_arc_in_rect_m
//                                  (length and first moment int y ds)
//   bil cx cy r x0 x1 y0 y1 bx by -> srt_arc_bilinear
// and prints one line per command, doubles in hex.  No CUDA call is made.
#include <stdio.h>
#include <string.h>

#include "common.cuh"

int main() {
  char op[16];
  while (scanf("%15s", op) == 1) {
    if (strcmp(op, "bf16") == 0) {
      double x;
      if (scanf("%la", &x) != 1) return 2;
      printf("%u\n", (unsigned)srt_f64_to_bf16(x));
    } else if (strcmp(op, "arc") == 0) {
      double a[7];
      for (int i = 0; i < 7; ++i)
        if (scanf("%la", &a[i]) != 1) return 2;
      double my = 0.0;
      const double len = srt_arc_in_rect(a[0], a[1], a[2], a[3], a[4], a[5], a[6]);
      const double len_m = srt_arc_in_rect_m(a[0], a[1], a[2], a[3], a[4], a[5], a[6], &my);
      printf("%a %a %a\n", len, len_m, my);
    } else if (strcmp(op, "bil") == 0) {
      double a[9];
      for (int i = 0; i < 9; ++i)
        if (scanf("%la", &a[i]) != 1) return 2;
      printf("%a\n", srt_arc_bilinear(a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7], a[8]));
    } else {
      return 3;
    }
  }
  return 0;
}
