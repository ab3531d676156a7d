"""GB300-native G1-G2 scheme: C-ABI library libg1g2 and its Python binding."""
