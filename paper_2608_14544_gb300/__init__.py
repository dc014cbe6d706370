"""GB300-native engine for momentum-jump-free mixed quantum-classical
Liouville dynamics (ensemble propagation behind a C ABI)."""
