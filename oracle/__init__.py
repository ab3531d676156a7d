"""CPU oracle of the G1-G2 scheme: test infrastructure only, never on the product path."""
