"""FP64 CPU oracle of the VP precoder (test infrastructure; never on the product path)."""
