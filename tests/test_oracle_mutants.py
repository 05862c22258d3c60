"""Plant plausible mistakes in copies of the oracle (on the CPU) and show that
at least one pin check fails for each, so the pins can catch such mistakes."""
from pathlib import Path

import pytest

import oracle
import pins

SRC = Path(oracle.__file__).resolve().parent / "oracle.c"

# (name, original text, mutated text): each is a mistake a careful reader could make.
MUTANTS = [
    ("mul_drops_carry_word", "wc[i + mb] = carry;", "wc[i + mb] = 0;"),
    ("mul_wrong_column", "u128 t = (u128)wa[i] * wb[j] + wc[i + j] + carry;",
     "u128 t = (u128)wa[i] * wb[j] + wc[i + j + (j == 1)] + carry;"),
    ("mul_skips_last_row", "for (uint32_t i = 0; i < ma; ++i) {", "for (uint32_t i = 0; i + 1 < ma; ++i) {"),
    ("add_loses_carry_in", "u128 s = (u128)wa[w] + wb[w] + carry;", "u128 s = (u128)wa[w] + wb[w];"),
    ("add_drops_top_limb", "from_u64(wc, n + 1, c);", "from_u64(wc, n, c); c[n] = 0;"),
    ("unpack_swaps_halves", "dst[k] = (uint32_t)(src[k / 2] >> (32 * (k % 2)));",
     "dst[k] = (uint32_t)(src[k / 2] >> (32 * (1 - k % 2)));"),
]


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, orig, bad):
    text = SRC.read_text()
    assert text.count(orig) == 1, "mutation anchor must be unique"
    src = tmp_path / f"{name}.c"
    src.write_text(text.replace(orig, bad))
    lib = oracle.OracleLib(oracle.compile_library(src, tmp_path / f"lib{name}.so"))
    caught = []
    for check in pins.ALL_CHECKS:
        try:
            check(lib)
        except AssertionError:
            caught.append(check.__name__)
    assert caught, f"no pin caught mutant {name}"
