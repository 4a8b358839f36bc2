"""GB300-native exact best-match subsequence search under banded DTW."""
